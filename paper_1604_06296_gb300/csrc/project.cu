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
// convention).  Three kernels compute the keys and the terms (term form):
//   bond_dft1, bond_dft2 -- F for every key (below)
//   contract_terms -- T and the basis change, per (target channel, 4 l)
// In a flow of a point-group covariant state the state is kept at the
// representative l of the loop rows only (wedge layout [3][nrow][nff][nff]):
// the Fourier keys still sum over every l, read through the signed
// permutation that maps each l to its row, and the last step runs at the
// representatives, writing the couplings in the wedge layout.
// The phase e^{i l.Y} is the only l dependence of a term, and the terms of a
// target channel take few distinct Y (41 at Nb = 13, 81 at Nb = 25), so the
// sums regroup (exactly, by linearity) as
//
//   V^T_mn(l) = V0_T + own_T + (1/Nl) Re sum_Y e^{i l.Y} H^T_mn(Y),
//   H^T_mn(Y) = sum_{b1,b2} c_m(b1) c_n(b2) G^T_{b1 b2}(Y),
//   G^T_{b1 b2}(Y) = sum_{terms of (b1, b2) at Y} sign * F_key,
//
// with G and H independent of l (grouped form).  It replaces contract_terms by
//   overlap   -- G and the basis change to H, per (target channel, Y)
//   contract  -- the phase sum over Y, a tiled complex matrix product
// and needs about half the arithmetic.  Views with a point of Nff >= 21 use
// it (there the sums bound the step); for Nff <= 13 its extra dependent
// launch costs more than the arithmetic it saves.
// The arithmetic type is FP64 for an FP64 context (this step is then bound by
// GB300's FP64 rate) and FP32 for the mixed-precision contexts, whose loops
// run on the tensor cores.  State and couplings are read and written in the
// arithmetic type: the FP32 kernels take an FP32 copy of the FP64 state (made
// by the flow's stage combination, or converted once per call) and write
// FP32 couplings (no FP64 conversion in them: GB300 converts between FP64
// and FP32 on its FP64 pipe, at a small fraction of the FP32 rate).
#include "device_util.cuh"

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
// acc + q * b for a complex q and a real b (paired FP32: one instruction)
__device__ __forceinline__ float2 cfma_real(float2 q, float b, float2 acc) {
  return fma2(q, make_float2(b, b), acc);
}
__device__ __forceinline__ double2 cfma_real(double2 q, double b, double2 acc) {
  return {fma(q.x, b, acc.x), fma(q.y, b, acc.y)};
}
template <class V>
__device__ __forceinline__ V to_c(double2 d) {
  return {(decltype(V::x))d.x, (decltype(V::x))d.y};
}

// bond coefficients and phase tables in the arithmetic type (FP32 copies
// made at setup: no FP64 conversions in the FP32 kernels)
__device__ __forceinline__ double2 coef_at(const PointDesc& pd, int e, double) {
  return pd.coef[e];
}
__device__ __forceinline__ float2 coef_at(const PointDesc& pd, int e, float) {
  return pd.coef_f[e];
}
__device__ __forceinline__ double2 phase_at(const PointDesc& pd, int e, double) {
  return pd.phase[e];
}
__device__ __forceinline__ float2 phase_at(const PointDesc& pd, int e, float) {
  return pd.phase_f[e];
}
__device__ __forceinline__ double2 yphase_at(const PointDesc& pd, size_t e, double) {
  return pd.yphase[e];
}
__device__ __forceinline__ float2 yphase_at(const PointDesc& pd, size_t e, float) {
  return pd.yphase_f[e];
}

// H(Y) rows [nff * nff] are stored with an even stride, so that every row
// starts on a 16-byte boundary (16-byte asynchronous copies)
__host__ __device__ constexpr int hstride(int nff) { return (nff * nff + 1) & ~1; }

// Fourier values of the keys, in two passes (each key (source S, bonds b3,
// b4, position X) is F = sum_l' e^{i l'.X} Bt^S_{b3 b4}(l') with
// Bt = C^T B C, C[a][b] = c_a(b); by linearity F = (C^T Bh^S(X) C)_{b3 b4}
// with the state's own Fourier value Bh^S_ab(X) = sum_l' e^{i l'.X} B^S_ab(l'),
// and e^{i l'.X} = e^{i l'_x X_x} e^{i l'_y X_y} on the coarse grid):
//   bond_dft1 -- P1[S][ix][dy][ab] = sum_iy e^{i l_y(iy) Y_dy} B^S_ab(ix, iy)
//   bond_dft2 -- Bh(X) = sum_ix e^{i l_x(ix) X_dx} P1[S][ix][dy][.], then
//                F[S][dx][dy][b3 b4] = (C^T Bh(X) C)_{b3 b4}
// The keys are numbered densely over (S, dx, dy, b3 b4): the X of all keys
// lie on a grid of nd x nd half-integer positions (nd = 9 for Nff = 13..25
// on grids of 16 or more points per direction).
constexpr int kDft1Threads = 128;
constexpr int kNdPass = 9;

// kWedge: the state is given at the rows' representatives only (wedge
// layout [3][nrow][nff][nff]); B(l) = R^g B(l0) R^g^T is read through the
// (row, g) serving l, (R^g X R^g^T)_ab = s_a s_b X_{p(a) p(b)}.
template <class T, bool kWedge>
__global__ void __launch_bounds__(kDft1Threads)
    bond_dft1_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix, int np,
                     const T* __restrict__ ybase, typename C2<T>::type* __restrict__ p1base) {
  using V = typename C2<T>::type;
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nff = pd.nff, nff2 = nff * nff, nd = pd.nd, ncx = pd.ncx, ncy = pd.ncy;
  const int chunks = (nff2 + kDft1Threads - 1) / kDft1Threads;
  const int loc = blockIdx.x - prefix[p];
  const int chunk = loc % chunks, rest = loc / chunks, ix = rest % ncx, src = rest / ncx;
  extern __shared__ double2 sm2[];
  V* ph = reinterpret_cast<V*>(sm2);  // [ncy][nd] e^{i l_y Y}
  for (int e = threadIdx.x; e < ncy * nd; e += blockDim.x)
    ph[e] = phase_at(pd, (ncx + e / nd) * nd + e % nd, T());
  // wedge: per iy the element offset of the serving row and its g; per g
  // and thread the signed offset + 1 of the thread's entry in the row
  int2* wr = reinterpret_cast<int2*>(ph + ncy * nd);  // [ncy]
  int* toff = reinterpret_cast<int*>(wr + ncy);       // [8][kDft1Threads]
  const int ab = chunk * kDft1Threads + threadIdx.x;
  if (kWedge) {
    for (int iy = threadIdx.x; iy < ncy; iy += blockDim.x) {
      const int2 rg = pd.lrow[ix * ncy + iy];
      wr[iy] = make_int2((src * pd.nrow + rg.x) * nff2, rg.y);
    }
    if (ab < nff2) {  // read back by this thread only
      const int a = ab / nff, b = ab - a * nff;
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        const int o = __ldg(pd.symperm + g * nff + a) * nff + __ldg(pd.symperm + g * nff + b) + 1;
        const int sg = __ldg(pd.symsign + g * nff + a) * __ldg(pd.symsign + g * nff + b);
        toff[g * kDft1Threads + threadIdx.x] = sg > 0 ? o : -o;
      }
    }
  }
  __syncthreads();
  if (ab >= nff2) return;
  const T* B = kWedge ? ybase + pd.off_wstate
                           : ybase + pd.off_state +
                                 ((size_t)src * pd.nl + (size_t)ix * ncy) * nff2 + ab;
  V* out = p1base + pd.off_bt + ((size_t)(src * ncx + ix) * nd) * nff2 + ab;
  // positions in passes of kNdPass (one pass for the bases of complete shells
  // on grids that resolve them; small grids alias more bond sums to more X);
  // the state in batches of kIyBatch rows, all loads of a batch in flight
  // before its arithmetic
  constexpr int kIyBatch = 16;
  for (int d0 = 0; d0 < nd; d0 += kNdPass) {
    V acc[kNdPass];
#pragma unroll
    for (int d = 0; d < kNdPass; ++d) acc[d] = {0, 0};
    for (int iy0 = 0; iy0 < ncy; iy0 += kIyBatch) {
      T bv[kIyBatch];
#pragma unroll
      for (int u = 0; u < kIyBatch; ++u) {
        const int iy = iy0 + u;
        bv[u] = 0;
        if (iy < ncy) {
          if (kWedge) {
            const int2 rg = wr[iy];
            const int o = toff[rg.y * kDft1Threads + threadIdx.x];
            const T w = __ldg(B + rg.x + abs(o) - 1);
            bv[u] = o > 0 ? w : -w;
          } else {
            bv[u] = __ldg(B + (size_t)iy * nff2);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kIyBatch; ++u) {
        if (iy0 + u >= ncy) break;
        const V* q = ph + (iy0 + u) * nd + d0;
#pragma unroll
        for (int d = 0; d < kNdPass; ++d)
          if (d0 + d < nd) acc[d] = cfma_real(q[d], bv[u], acc[d]);
      }
    }
#pragma unroll
    for (int d = 0; d < kNdPass; ++d)
      if (d0 + d < nd) out[(size_t)(d0 + d) * nff2] = acc[d];
  }
}

// Fourier values of the keys of one (source, X) from the state's DFT Bh(X)
// (after a barrier): F = C^T Bh C, C[a][b] = c_a(b), through tmp [nff][nb]
// (a barrier in between).
template <class V>
__device__ __forceinline__ void keys_from_bh(const V* cs, const V* Bh, V* tmp, int nff, int nb,
                                             V* F) {
  // tmp[a][b4] = sum_b Bh[a][b] c_b(b4)
  for (int e = threadIdx.x; e < nff * nb; e += blockDim.x) {
    const int a = e / nb, b4 = e - a * nb;
    V acc = {0, 0};
    for (int b = 0; b < nff; ++b) acc = cfma(Bh[a * nff + b], cs[b * nb + b4], acc);
    tmp[e] = acc;
  }
  __syncthreads();
  // F[b3][b4] = sum_a c_a(b3) tmp[a][b4]
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int b3 = e / nb, b4 = e - b3 * nb;
    V acc = {0, 0};
    for (int a = 0; a < nff; ++a) acc = cfma(cs[a * nb + b3], tmp[a * nb + b4], acc);
    F[e] = acc;
  }
}

template <class T, int NF>
__global__ void __launch_bounds__(256)
    bond_dft2_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix, int np,
                     const typename C2<T>::type* __restrict__ p1base,
                     typename C2<T>::type* __restrict__ fkbase) {
  using V = typename C2<T>::type;
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nff = NF ? NF : pd.nff, nb = NF ? NF : pd.nb, nff2 = nff * nff;
  const int nd = pd.nd, ncx = pd.ncx;
  const int loc = blockIdx.x - prefix[p];
  const int dy = loc % nd, dx = (loc / nd) % nd, src = loc / (nd * nd);
  extern __shared__ double2 sm2[];
  V* cs = reinterpret_cast<V*>(sm2);  // [nff][nb]
  V* Bh = cs + nff * nb;              // [nff][nff]
  V* tmp = Bh + nff2;                 // [nff][nb]
  V* phx = tmp + nff * nb;            // [ncx] e^{i l_x X}
  for (int e = threadIdx.x; e < nff * nb; e += blockDim.x) cs[e] = coef_at(pd, e, T());
  for (int e = threadIdx.x; e < ncx; e += blockDim.x) phx[e] = phase_at(pd, e * nd + dx, T());
  __syncthreads();
  const size_t xstride = (size_t)nd * nff2;
  const V* P1 = p1base + pd.off_bt + (size_t)dy * nff2 + (size_t)src * ncx * xstride;
  // the entries ab = threadIdx.x + r * 256 of this thread, in batches of kXB
  // positions ix with all kR * kXB loads in flight before the arithmetic
  {
    constexpr int kR = (kMaxNf * kMaxNf + 255) / 256;
    constexpr int kXB = sizeof(T) == 4 ? 8 : 4;
    V acc[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) acc[r] = {0, 0};
    for (int ix0 = 0; ix0 < ncx; ix0 += kXB) {
      V q[kR][kXB];
#pragma unroll
      for (int r = 0; r < kR; ++r)
#pragma unroll
        for (int u = 0; u < kXB; ++u) {
          const int ab = threadIdx.x + 256 * r, ix = ix0 + u;
          q[r][u] = ab < nff2 && ix < ncx ? P1[(size_t)ix * xstride + ab] : V{0, 0};
        }
#pragma unroll
      for (int u = 0; u < kXB; ++u) {
        if (ix0 + u >= ncx) break;
        const V e = phx[ix0 + u];
#pragma unroll
        for (int r = 0; r < kR; ++r) acc[r] = cfma(e, q[r][u], acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < kR; ++r)
      if (threadIdx.x + 256 * r < nff2) Bh[threadIdx.x + 256 * r] = acc[r];
  }
  __syncthreads();
  keys_from_bh(cs, Bh, tmp, nff, nb,
               fkbase + pd.off_fkey + ((size_t)(src * nd + dx) * nd + dy) * nb * nb);
}

// Non-uniform meshes: the Fourier values of the keys as quadratures over the
// source channel's mesh, Bh(X) = sum_{l'} E_S(X, l') B^S(l') with the
// scale-independent E_S(X, l') = nl w_S(l') e^{i l'.X} (the factor nl undoes
// the phase sums' 1/nl; P's weights for S = P, mesh_CD's for C and D), then
// F = C^T Bh(X) C -- a complex-by-real matrix product over the mesh points,
// split over chunks of points (E stored point-major, [2][nl][nd^2]):
//   mesh_dft_partial -- per (source, chunk, tile of 64 entries ab): the partial
//     sums of every position X over the chunk's points, staged kMeshSub points
//     at a time in shared memory; thread: kXT adjacent positions x 4 adjacent
//     entries;
//   mesh_dft_reduce  -- per (source, X): the chunks' sum in a fixed order, then
//     the basis change.
// kWedge: the state is given at the rows' representatives only and B(l) =
// R^g B(l0) R^g^T is read through the (row, g) serving l, as in bond_dft1.
constexpr int kMeshSub = 32;

__host__ __device__ inline int mesh_ab_tiles(int nff) { return (nff * nff + kMeshAB - 1) / kMeshAB; }

template <class T>
__device__ __forceinline__ const typename C2<T>::type* mesh_e_of(const PointDesc& pd);
template <>
__device__ __forceinline__ const double2* mesh_e_of<double>(const PointDesc& pd) {
  return pd.mesh_e;
}
template <>
__device__ __forceinline__ const float2* mesh_e_of<float>(const PointDesc& pd) {
  return pd.mesh_e_f;
}

template <class T, int kXT, bool kWedge>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
    mesh_dft_partial_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix,
                            int np, const T* __restrict__ ybase,
                            typename C2<T>::type* __restrict__ pbase) {
  using V = typename C2<T>::type;
  constexpr int kXP = 16 * kXT;  // positions per CTA (padded)
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nff = pd.nff, nff2 = nff * nff, nx = pd.nd * pd.nd, nl = pd.nl;
  const int tiles = mesh_ab_tiles(nff), chunks = pd.mesh_chunks;
  const int loc = blockIdx.x - prefix[p];
  const int tile = loc % tiles, chunk = (loc / tiles) % chunks, src = loc / (tiles * chunks);
  const int ab0 = tile * kMeshAB;
  const int l0 = chunk * pd.mesh_lc, l1 = min(nl, l0 + pd.mesh_lc);
  extern __shared__ double2 sm2[];
  V* Es = reinterpret_cast<V*>(sm2);                           // [kMeshSub][kXP]
  T* Bs = reinterpret_cast<T*>(Es + kMeshSub * kXP);           // [kMeshSub][kMeshAB]
  int* toff = reinterpret_cast<int*>(Bs + kMeshSub * kMeshAB);  // [8][kMeshAB] wedge
  const V* E = mesh_e_of<T>(pd) + (size_t)(src == 0 ? 0 : 1) * nx * nl;
  const T* B = kWedge ? ybase + pd.off_wstate : ybase + pd.off_state + (size_t)src * nl * nff2;
  if (kWedge)
    for (int e = threadIdx.x; e < 8 * kMeshAB; e += blockDim.x) {
      const int g = e / kMeshAB, ab = ab0 + e % kMeshAB;
      int o = 0;
      if (ab < nff2) {
        const int a = ab / nff, b = ab - a * nff;
        o = __ldg(pd.symperm + g * nff + a) * nff + __ldg(pd.symperm + g * nff + b) + 1;
        if (__ldg(pd.symsign + g * nff + a) * __ldg(pd.symsign + g * nff + b) < 0) o = -o;
      }
      toff[e] = o;
    }
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  V acc[kXT][4];
#pragma unroll
  for (int i = 0; i < kXT; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[i][k] = {0, 0};
  // a stage's operands are loaded into registers, then stored to shared
  // memory (kPre: during the previous stage's arithmetic; off: the registers
  // are better spent on two CTAs per SM, FP32, or the FP64 accumulators)
  constexpr bool kPre = sizeof(T) == 4;
  constexpr int kEPer = kMeshSub * kXP / 256, kBPer = kMeshSub * kMeshAB / 256;
  V ereg[kEPer];
  T breg[kBPer];
  auto fetch = [&](int ls) {
#pragma unroll
    for (int u = 0; u < kEPer; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int j = e / kXP, x = e % kXP;  // consecutive positions per point
      ereg[u] = x < nx && ls + j < l1 ? __ldg(E + (size_t)(ls + j) * nx + x) : V{0, 0};
    }
#pragma unroll
    for (int u = 0; u < kBPer; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int j = e / kMeshAB, c = e % kMeshAB, l = ls + j;
      T b = 0;
      if (l < l1 && ab0 + c < nff2) {
        if (kWedge) {
          const int2 rg = __ldg(pd.lrow + l);
          const int o = toff[rg.y * kMeshAB + c];
          const T v = __ldg(B + (size_t)(src * pd.nrow + rg.x) * nff2 + abs(o) - 1);
          b = o > 0 ? v : -v;
        } else {
          b = __ldg(B + (size_t)l * nff2 + ab0 + c);
        }
      }
      breg[u] = b;
    }
  };
  __syncthreads();  // toff written
  if (kPre && l0 < l1) fetch(l0);
  for (int ls = l0; ls < l1; ls += kMeshSub) {
    if (!kPre) fetch(ls);
    __syncthreads();  // the previous stage is consumed
#pragma unroll
    for (int u = 0; u < kEPer; ++u) {
      const int e = threadIdx.x + 256 * u;
      Es[e] = ereg[u];  // [j][x]: contiguous, conflict-free
    }
#pragma unroll
    for (int u = 0; u < kBPer; ++u) Bs[threadIdx.x + 256 * u] = breg[u];
    __syncthreads();
    if (kPre && ls + kMeshSub < l1) fetch(ls + kMeshSub);
#pragma unroll 2
    for (int j = 0; j < kMeshSub; ++j) {
      // the thread's kXT adjacent positions and 4 adjacent entries: 16-byte
      // shared-memory loads (the warp's two position slices are broadcasts)
      T bv[4];
      V ev[kXT];
      if constexpr (sizeof(T) == 4) {
        const float4 b4 = *reinterpret_cast<const float4*>(Bs + j * kMeshAB + 4 * tx);
        bv[0] = b4.x, bv[1] = b4.y, bv[2] = b4.z, bv[3] = b4.w;
        const float4* ep = reinterpret_cast<const float4*>(Es + j * kXP + kXT * ty);
#pragma unroll
        for (int i = 0; i < kXT / 2; ++i) {
          const float4 q = ep[i];
          ev[2 * i] = {q.x, q.y};
          ev[2 * i + 1] = {q.z, q.w};
        }
      } else {
        const double2* bp = reinterpret_cast<const double2*>(Bs + j * kMeshAB + 4 * tx);
        const double2 b0 = bp[0], b1 = bp[1];
        bv[0] = b0.x, bv[1] = b0.y, bv[2] = b1.x, bv[3] = b1.y;
#pragma unroll
        for (int i = 0; i < kXT; ++i) ev[i] = Es[j * kXP + kXT * ty + i];
      }
#pragma unroll
      for (int i = 0; i < kXT; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          acc[i][k].x = fma(ev[i].x, bv[k], acc[i][k].x);
          acc[i][k].y = fma(ev[i].y, bv[k], acc[i][k].y);
        }
      }
    }
  }
  V* out = pbase + pd.off_bt + (size_t)(src * chunks + chunk) * nx * nff2;
#pragma unroll
  for (int i = 0; i < kXT; ++i) {
    const int x = kXT * ty + i;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ab = ab0 + 4 * tx + k;
      if (x < nx && ab < nff2) out[(size_t)x * nff2 + ab] = acc[i][k];
    }
  }
}

template <class T, int NF>
__global__ void __launch_bounds__(256)
    mesh_dft_reduce_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix,
                           int np, const typename C2<T>::type* __restrict__ pbase,
                           typename C2<T>::type* __restrict__ fkbase) {
  using V = typename C2<T>::type;
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nff = NF ? NF : pd.nff, nb = NF ? NF : pd.nb, nff2 = nff * nff;
  const int nd = pd.nd, nx = nd * nd, chunks = pd.mesh_chunks;
  const int loc = blockIdx.x - prefix[p];
  const int x = loc % nx, src = loc / nx;
  extern __shared__ double2 sm2[];
  V* cs = reinterpret_cast<V*>(sm2);  // [nff][nb]
  V* Bh = cs + nff * nb;              // [nff][nff]
  V* tmp = Bh + nff2;                 // [nff][nb]
  for (int e = threadIdx.x; e < nff * nb; e += blockDim.x) cs[e] = coef_at(pd, e, T());
  const V* part = pbase + pd.off_bt + ((size_t)src * chunks * nx + x) * nff2;
  for (int ab = threadIdx.x; ab < nff2; ab += blockDim.x) {
    V acc = {0, 0};
    for (int c = 0; c < chunks; ++c) {
      const V v = part[(size_t)c * nx * nff2 + ab];
      acc.x += v.x;
      acc.y += v.y;
    }
    Bh[ab] = acc;
  }
  __syncthreads();
  keys_from_bh(cs, Bh, tmp, nff, nb, fkbase + pd.off_fkey + ((size_t)src * nx + x) * nb * nb);
}

// The tensor-core quadrature's partial products (FP32 [3][kz][mpad][npad],
// rows 2x and 2x + 1 the real and imaginary part of position x) added over
// the splits in a fixed order, then the basis change.  One CTA per (source, X).
template <int NF>
__global__ void __launch_bounds__(256)
    mesh_tc_reduce_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix,
                          int np, const float* __restrict__ part, float2* __restrict__ fkbase) {
  using V = float2;
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nff = NF ? NF : pd.nff, nb = NF ? NF : pd.nb, nff2 = nff * nff;
  const int nd = pd.nd, nx = nd * nd, kz = pd.mesh_kz, mpad = pd.mesh_mpad, npad = pd.mesh_npad;
  const int loc = blockIdx.x - prefix[p];
  const int x = loc % nx, src = loc / nx;
  extern __shared__ double2 sm2[];
  V* cs = reinterpret_cast<V*>(sm2);  // [nff][nb]
  V* Bh = cs + nff * nb;              // [nff][nff]
  V* tmp = Bh + nff2;                 // [nff][nb]
  for (int e = threadIdx.x; e < nff * nb; e += blockDim.x) cs[e] = coef_at(pd, e, float());
  const float* pr = part + (size_t)src * kz * mpad * npad + (size_t)(2 * x) * npad;
  for (int ab = threadIdx.x; ab < nff2; ab += blockDim.x) {
    V acc = {0.f, 0.f};
    for (int z = 0; z < kz; ++z) {
      const float* q = pr + (size_t)z * mpad * npad + ab;
      acc.x += q[0];
      acc.y += q[npad];
    }
    Bh[ab] = acc;
  }
  __syncthreads();
  keys_from_bh(cs, Bh, tmp, nff, nb, fkbase + pd.off_fkey + ((size_t)src * nx + x) * nb * nb);
}

// Element offset of the state and couplings of channel t at output slot q
// (transfer momentum l): l in the full layout, or row q in the wedge layout.
__device__ __forceinline__ size_t slot_offset(const PointDesc& pd, int rows, int t, int q, int l,
                                              int n2) {
  return rows ? pd.off_wstate + ((size_t)t * pd.nrow + q) * n2
              : pd.off_state + ((size_t)t * pd.nl + l) * n2;
}

// Term form (Nff <= 13).  kTermsL transfer momenta of one target channel per
// CTA: each term of the (scale-independent) overlap lists and its Fourier key
// are read once and applied to all of them (only the phases e^{i l.Y} differ).
constexpr int kTermsL = 4;
constexpr int kTermBatch = 8;

template <class T, int NF>
__global__ void __launch_bounds__(256)
    contract_terms_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix, int np,
                    const T* __restrict__ ybase,
                    const typename C2<T>::type* __restrict__ fkbase, T* __restrict__ vbase,
                    int rows) {
  using V = typename C2<T>::type;
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nb = NF ? NF : pd.nb, nff = NF ? NF : pd.nff, nl = pd.nl, nd = pd.nd;
  // output slots: every l, or the representative l of every loop row
  const int nout = rows ? pd.nrow : nl;
  const int groups = (nout + kTermsL - 1) / kTermsL;
  const int loc = blockIdx.x - prefix[p];
  const int t = loc / groups, q0 = (loc % groups) * kTermsL;
  const int nlb = min(kTermsL, nout - q0);  // slots of this CTA
  __shared__ int sl[kTermsL];               // l of each slot (the last one repeated)
  if (threadIdx.x < kTermsL) {
    const int q = q0 + min((int)threadIdx.x, nlb - 1);
    sl[threadIdx.x] = rows ? pd.rowimg[pd.rowimg_ptr[q]].x : q;
  }
  __syncthreads();
  extern __shared__ double2 sm2[];
  V* Tm = reinterpret_cast<V*>(sm2);       // [kTermsL][nb][nb]
  V* tmp = Tm + kTermsL * nb * nb;      // [kTermsL][nb][nff]
  V* cs = tmp + kTermsL * nb * nff;     // [nff][nb]
  V* qx = cs + nff * nb;                   // [kTermsL][nd]
  V* qy = qx + kTermsL * nd;            // [kTermsL][nd]
  const size_t n2 = (size_t)nff * nff;
  const T own_sign = t == 0 ? -1 : 1;  // V^P = V0 - P + ...; V^C = V0 + C + ...
  const T U = (T)pd.U;
  if (!pd.feedback) {
    for (int e = threadIdx.x; e < nlb * (int)n2; e += blockDim.x) {
      const int j = e / (int)n2, r = e % (int)n2;
      const size_t o = slot_offset(pd, rows, t, q0 + j, sl[j], (int)n2) + r;
      vbase[o] = (r == 0 ? U : T(0)) + own_sign * ybase[o];
    }
    return;
  }
  for (int e = threadIdx.x; e < nff * nb; e += blockDim.x) cs[e] = coef_at(pd, e, T());
  for (int e = threadIdx.x; e < kTermsL * nd; e += blockDim.x) {
    const int j = e / nd, d = e % nd;
    const int l = sl[j];
    const int ix = l / pd.ncy, iy = l - ix * pd.ncy;
    qx[e] = phase_at(pd, ix * nd + d, T());
    qy[e] = phase_at(pd, (pd.ncx + iy) * nd + d, T());
  }
  __syncthreads();
  const int* rp = pd.row_ptr + (size_t)t * (nb * nb + 1);
  const int4* tm = pd.terms + pd.term_off[t];
  const V* fkey = fkbase + pd.off_fkey;
  const T inv_nl = T(1) / T(nl);
  for (int o = threadIdx.x; o < nb * nb; o += blockDim.x) {
    V acc[kTermsL];
#pragma unroll
    for (int j = 0; j < kTermsL; ++j) acc[j] = {0, 0};
    // terms in batches of kTermBatch: all terms of a batch, then all their
    // keys, are loaded before any is used (rows hold up to ~26 terms, and the
    // key loads depend on the term loads)
    const int ke = rp[o + 1];
    for (int k = rp[o]; k < ke; k += kTermBatch) {
      int4 q[kTermBatch];
      V f[kTermBatch];
#pragma unroll
      for (int i = 0; i < kTermBatch; ++i) q[i] = k + i < ke ? tm[k + i] : make_int4(0, 0, 0, 0);
#pragma unroll
      for (int i = 0; i < kTermBatch; ++i) {
        f[i] = k + i < ke ? fkey[q[i].x] : V{0, 0};
        if (q[i].w < 0) f[i] = {-f[i].x, -f[i].y};
      }
#pragma unroll
      for (int i = 0; i < kTermBatch; ++i)
#pragma unroll
        for (int j = 0; j < kTermsL; ++j)
          acc[j] = cfma(cmul(qx[j * nd + q[i].y], qy[j * nd + q[i].z]), f[i], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < kTermsL; ++j) Tm[j * nb * nb + o] = {acc[j].x * inv_nl, acc[j].y * inv_nl};
  }
  __syncthreads();
  // basis change for all l of the CTA at once: rows of cw lanes (lane n <
  // nff is column n), 32 / cw rows per warp, the kTermsL l of a row in
  // one thread (independent chains, each coefficient read once)
  const int cw = nff <= 16 ? 16 : 32, rpw = 32 / cw;
  const int lane = threadIdx.x & 31, n = lane & (cw - 1);
  const int r0 = (threadIdx.x >> 5) * rpw + lane / cw, rstep = (blockDim.x >> 5) * rpw;
  // tmp[j][b1][n] = sum_b2 T_j[b1][b2] c_n(b2)
  for (int b1 = r0; b1 < nb; b1 += rstep) {
    if (n >= nff) continue;
    V acc[kTermsL];
#pragma unroll
    for (int jj = 0; jj < kTermsL; ++jj) acc[jj] = {0, 0};
    for (int b2 = 0; b2 < nb; ++b2) {
      const V c = cs[n * nb + b2];
#pragma unroll
      for (int jj = 0; jj < kTermsL; ++jj)
        acc[jj] = cfma(Tm[jj * nb * nb + b1 * nb + b2], c, acc[jj]);
    }
#pragma unroll
    for (int jj = 0; jj < kTermsL; ++jj) tmp[(jj * nb + b1) * nff + n] = acc[jj];
  }
  __syncthreads();
  // V_mn = V0 + own + Re sum_b1 c_m(b1) tmp[b1][n]
  for (int m = r0; m < nff; m += rstep) {
    if (n >= nff) continue;
    const int mn = m * nff + n;
    T yv[kTermsL];
#pragma unroll
    for (int jj = 0; jj < kTermsL; ++jj)
      yv[jj] = jj < nlb ? ybase[slot_offset(pd, rows, t, q0 + jj, sl[jj], n2) + mn] : T(0);
    T acc[kTermsL];
#pragma unroll
    for (int jj = 0; jj < kTermsL; ++jj) acc[jj] = 0;
    for (int b1 = 0; b1 < nb; ++b1) {
      const V c1 = cs[m * nb + b1];
#pragma unroll
      for (int jj = 0; jj < kTermsL; ++jj) {
        const V t1 = tmp[(jj * nb + b1) * nff + n];
        acc[jj] = fma(c1.x, t1.x, fma(-c1.y, t1.y, acc[jj]));  // real part of c * tmp
      }
    }
#pragma unroll
    for (int jj = 0; jj < kTermsL; ++jj)
      if (jj < nlb)
        vbase[slot_offset(pd, rows, t, q0 + jj, sl[jj], n2) + mn] =
            (mn == 0 ? U : T(0)) + own_sign * yv[jj] + acc[jj];
  }
}

// Grouped form (Nff >= 21).  One CTA per (target channel, phase position Y):
// G(Y) from the keys of its terms, then H(Y) = c^T G(Y) c, written over the
// point's bond-space workspace (the bond-space propagators are no longer
// needed once the keys exist).  Every thread loads one term slot and its key
// at once (two round trips); the first term of each output pair then adds
// its pair's terms in slot order.
template <class T, int NF>
__global__ void __launch_bounds__(256)
    overlap_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix, int np,
                   const typename C2<T>::type* __restrict__ fkbase,
                   typename C2<T>::type* __restrict__ hbase) {
  using V = typename C2<T>::type;
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nb = NF ? NF : pd.nb, nff = NF ? NF : pd.nff;
  const int g = blockIdx.x - prefix[p];  // over the positions of all three targets
  const int nt = pd.gmaxt;
  extern __shared__ double2 sm2[];
  V* G = reinterpret_cast<V*>(sm2);  // [nb][nb]
  V* tmp = G + nb * nb;              // [nb][nff]
  V* cs = tmp + nb * nff;            // [nff][nb]
  V* tv = cs + nff * nb;             // [nt] signed key values
  int* to = reinterpret_cast<int*>(tv + nt);  // [nt] output pair of each slot (-1: unused)
  const int4* slot = pd.gslot + (size_t)g * nt;
  const V* fkey = fkbase + pd.off_fkey;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    const int4 q = slot[k];
    V f = {0, 0};
    if (q.y >= 0) f = fkey[q.y];
    tv[k] = q.z < 0 ? V{-f.x, -f.y} : f;
    to[k] = q.x;
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) G[e] = {0, 0};
  for (int e = threadIdx.x; e < nff * nb; e += blockDim.x) cs[e] = coef_at(pd, e, T());
  __syncthreads();
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    const int o = to[k];
    if (o < 0 || (k > 0 && to[k - 1] == o)) continue;
    V acc = tv[k];
    for (int k2 = k + 1; k2 < nt && to[k2] == o; ++k2) {
      acc.x += tv[k2].x;
      acc.y += tv[k2].y;
    }
    G[o] = acc;
  }
  __syncthreads();
  // tmp[b1][n] = sum_b2 G[b1][b2] c_n(b2)
  for (int e = threadIdx.x; e < nb * nff; e += blockDim.x) {
    const int b1 = e / nff, n = e - b1 * nff;
    V acc = {0, 0};
    for (int b2 = 0; b2 < nb; ++b2) acc = cfma(G[b1 * nb + b2], cs[n * nb + b2], acc);
    tmp[e] = acc;
  }
  __syncthreads();
  // H[m][n] = sum_b1 c_m(b1) tmp[b1][n]
  V* H = hbase + pd.off_bt + (size_t)g * hstride(nff);
  for (int e = threadIdx.x; e < nff * nff; e += blockDim.x) {
    const int m = e / nff, n = e - m * nff;
    V acc = {0, 0};
    for (int b1 = 0; b1 < nb; ++b1) acc = cfma(cs[m * nb + b1], tmp[b1 * nff + n], acc);
    H[e] = acc;
  }
}

// The phase sums of the grouped form as a tiled complex matrix product:
//   V(l)_mn = V0 + own + (1/Nl) Re sum_Y E[l][Y] H[Y][mn],  E[l][Y] = e^{i l.Y}
// over the output slots (every l, or the rows' representatives) and the
// Nff^2 entries, the positions Y of the target as the contraction index.
// CTA: (point, target, kCL slots, kCM entries); positions in passes (32 in
// FP32, 16 in FP64: 37 KB of static shared memory), staged with E in shared
// memory; thread: one entry, kCR slots.
constexpr int kCL = 16;      // output slots per CTA
constexpr int kCM = 128;     // entries (m, n) per CTA
constexpr int kCYBytes = 32 * 8;  // positions per pass x bytes per complex value
constexpr int kCThreads = 256;
constexpr int kCR = kCL * kCM / kCThreads;  // slots per thread (8)

__host__ __device__ inline int contract_ctiles(int nout, int nff) {
  return ((nout + kCL - 1) / kCL) * ((nff * nff + kCM - 1) / kCM);
}

template <class T, int NF>
__global__ void __launch_bounds__(kCThreads)
    contract_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix, int np,
                    const T* __restrict__ ybase,
                    const typename C2<T>::type* __restrict__ hbase, T* __restrict__ vbase,
                    int rows) {
  using V = typename C2<T>::type;
  constexpr int kCY = kCYBytes / (int)sizeof(V);
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nff = NF ? NF : pd.nff, nl = pd.nl, n2 = nff * nff, n2p = hstride(nff);
  const int nout = rows ? pd.nrow : nl;
  const int tiles = contract_ctiles(nout, nff), mtiles = (n2 + kCM - 1) / kCM;
  const int loc = blockIdx.x - prefix[p];
  const int t = loc / tiles, r = loc % tiles;
  const int q0 = (r / mtiles) * kCL, mn0 = (r % mtiles) * kCM;
  const int nlb = min(kCL, nout - q0);  // slots of this CTA
  __shared__ int sl[kCL];  // l of each slot (the last one repeated)
  // e^{i l.Y} of a pass: FP32 as two planes per position (Re, then -Im) for
  // the paired arithmetic; FP64 as complex values
  __shared__ __align__(16) V Es[kCY][kCL];
  __shared__ __align__(16) V Hs[kCY][kCM];  // H of a pass
  if (threadIdx.x < kCL) {
    const int q = q0 + min((int)threadIdx.x, nlb - 1);
    sl[threadIdx.x] = rows ? pd.rowimg[pd.rowimg_ptr[q]].x : q;
  }
  __syncthreads();
  const T own_sign = t == 0 ? -1 : 1;  // V^P = V0 - P + ...; V^C = V0 + C + ...
  const T U = (T)pd.U;
  const int c = threadIdx.x % kCM, j0 = (threadIdx.x / kCM) * kCR;  // entry, first slot
  const int mn = mn0 + c;
  T acc[kCR];
#pragma unroll
  for (int j = 0; j < kCR; ++j) acc[j] = 0;
  if (pd.feedback) {
    const int y0 = pd.gy_off[t], ny = pd.gy_off[t + 1] - y0;
    const V* H = hbase + pd.off_bt + (size_t)y0 * n2p;
    // a pass's operands are loaded into registers during the previous pass's
    // arithmetic, then stored to shared memory
    constexpr int kHPer = kCY * kCM / kCThreads, kEPer = (kCY * kCL + kCThreads - 1) / kCThreads;
    V hreg[kHPer], ereg[kEPer];
    auto fetch = [&](int c0) {
      const int cn = min(kCY, ny - c0);
#pragma unroll
      for (int u = 0; u < kHPer; ++u) {
        const int e = threadIdx.x + u * kCThreads, yi = e / kCM, cc = e % kCM;
        hreg[u] = yi < cn && mn0 + cc < n2 ? H[(size_t)(c0 + yi) * n2p + mn0 + cc] : V{0, 0};
      }
#pragma unroll
      for (int u = 0; u < kEPer; ++u) {
        const int e = threadIdx.x + u * kCThreads, yi = e / kCL, j = e % kCL;
        ereg[u] = e < kCY * kCL && yi < cn
                      ? yphase_at(pd, (size_t)(y0 + c0 + yi) * nl + sl[j], T())
                      : V{0, 0};
      }
    };
    if (ny > 0) fetch(0);
    for (int c0 = 0; c0 < ny; c0 += kCY) {
      __syncthreads();  // the previous pass is consumed
#pragma unroll
      for (int u = 0; u < kHPer; ++u) {
        const int e = threadIdx.x + u * kCThreads;
        Hs[e / kCM][e % kCM] = hreg[u];
      }
#pragma unroll
      for (int u = 0; u < kEPer; ++u) {
        const int e = threadIdx.x + u * kCThreads, yi = e / kCL, j = e % kCL;
        if (e < kCY * kCL) {
          if constexpr (sizeof(T) == 4) {
            float* row = reinterpret_cast<float*>(&Es[yi][0]);
            row[j] = ereg[u].x;
            row[kCL + j] = -ereg[u].y;
          } else {
            Es[yi][j] = ereg[u];
          }
        }
      }
      __syncthreads();
      if (c0 + kCY < ny) fetch(c0 + kCY);
      if constexpr (sizeof(T) == 4) {
        // slots in pairs: acc(j, j + 1) += (-Im e) Im h, then += (Re e) Re h
        // (each lane takes the two roundings of the scalar form)
        float2 a2[kCR / 2];
#pragma unroll
        for (int j = 0; j < kCR / 2; ++j) a2[j] = make_float2(acc[2 * j], acc[2 * j + 1]);
#pragma unroll 4
        for (int yi = 0; yi < kCY; ++yi) {
          const V h = Hs[yi][c];
          const float2 hx = make_float2(h.x, h.x), hy = make_float2(h.y, h.y);
          const float* row = reinterpret_cast<const float*>(&Es[yi][0]);
#pragma unroll
          for (int j = 0; j < kCR; j += 4) {
            const float4 ex = *reinterpret_cast<const float4*>(row + j0 + j);
            const float4 ey = *reinterpret_cast<const float4*>(row + kCL + j0 + j);
            a2[j / 2] = fma2(make_float2(ey.x, ey.y), hy, a2[j / 2]);
            a2[j / 2] = fma2(make_float2(ex.x, ex.y), hx, a2[j / 2]);
            a2[j / 2 + 1] = fma2(make_float2(ey.z, ey.w), hy, a2[j / 2 + 1]);
            a2[j / 2 + 1] = fma2(make_float2(ex.z, ex.w), hx, a2[j / 2 + 1]);
          }
        }
#pragma unroll
        for (int j = 0; j < kCR / 2; ++j) {
          acc[2 * j] = a2[j].x;
          acc[2 * j + 1] = a2[j].y;
        }
      } else {
#pragma unroll 4
        for (int yi = 0; yi < kCY; ++yi) {
          const V h = Hs[yi][c];
#pragma unroll
          for (int j = 0; j < kCR; ++j) {
            const V e = Es[yi][j0 + j];
            acc[j] = fma(e.x, h.x, fma(-e.y, h.y, acc[j]));  // real part of e * h
          }
        }
      }
    }
  }
  if (mn >= n2) return;
  const T inv_nl = T(1) / T(nl);
#pragma unroll
  for (int j = 0; j < kCR; ++j)
    if (j0 + j < nlb) {
      const size_t o = slot_offset(pd, rows, t, q0 + j0 + j, sl[j0 + j], n2) + mn;
      vbase[o] = (mn == 0 ? U : T(0)) + own_sign * ybase[o] + acc[j] * inv_nl;
    }
}

template <class T>
size_t dft1_smem(const MultiView& v) {
  size_t m = 1;
  for (const PointDesc& d : v.h)
    m = std::max(m, sizeof(typename C2<T>::type) * d.ncy * d.nd + sizeof(int2) * d.ncy +
                        sizeof(int) * 8 * kDft1Threads);
  return m;
}
template <class T>
size_t dft2_smem(const MultiView& v) {
  int m = 1;
  for (const PointDesc& d : v.h) m = std::max(m, d.ncx);
  return sizeof(typename C2<T>::type) *
         (2 * (size_t)v.nff_max * v.nb_max + (size_t)v.nff_max * v.nff_max + m);
}
// positions per thread of the mesh partial sums (16 threads per position
// column): 6 up to 96 positions, 8 up to 128 (nd <= 11)
int mesh_xt(const MultiView& v) {
  int nx = 0;
  for (const PointDesc& d : v.h) nx = std::max(nx, d.nd * d.nd);
  return nx <= 96 ? 6 : 8;
}
template <class T>
size_t mesh_partial_smem(int xt) {
  return sizeof(typename C2<T>::type) * kMeshSub * 16 * xt + sizeof(T) * kMeshSub * kMeshAB +
         sizeof(int) * 8 * kMeshAB;
}
template <class T>
size_t mesh_reduce_smem(const MultiView& v) {
  return sizeof(typename C2<T>::type) *
         (2 * (size_t)v.nff_max * v.nb_max + (size_t)v.nff_max * v.nff_max);
}
template <class T>
size_t overlap_smem(const MultiView& v) {
  int nt = 1;
  for (const PointDesc& d : v.h) nt = std::max(nt, d.gmaxt);
  return sizeof(typename C2<T>::type) *
             ((size_t)v.nb_max * v.nb_max + 2 * (size_t)v.nb_max * v.nff_max + nt) +
         sizeof(int) * (size_t)nt;
}

template <class T>
size_t contract_terms_smem(const MultiView& v) {
  return sizeof(typename C2<T>::type) *
         ((size_t)kTermsL * v.nb_max * v.nb_max + (kTermsL + 1) * (size_t)v.nb_max * v.nff_max +
          2 * (size_t)kTermsL * v.nd_max);
}

// the largest dynamic shared memory a kernel may take: the device limit less
// its static shared memory
template <class K>
cudaError_t allow_dynamic_smem(K* kernel, int optin) {
  cudaFuncAttributes a{};
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)a.sharedSizeBytes);
}

template <class T>
tufrg_status prepare_typed(const MultiView& v) {
  const int smem = smem_optin();
  // (the two contract kernels also hold a few bytes of static shared memory)
  if ((int)dft1_smem<T>(v) > smem || (int)dft2_smem<T>(v) > smem ||
      (int)mesh_partial_smem<T>(8) > smem ||
      (int)overlap_smem<T>(v) > smem ||
      (int)contract_terms_smem<T>(v) + 64 > smem)
    return TUFRG_ERR_ARG;
  if (v.mesh) {
    int nx = 0;
    for (const PointDesc& d : v.h) nx = std::max(nx, d.nd * d.nd);
    if (nx > 128) return TUFRG_ERR_ARG;
    TUFRG_CHECK(prepare_mesh_tc());
  }
  TUFRG_CUDA(cudaFuncSetAttribute(mesh_dft_partial_kernel<T, 6, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  TUFRG_CUDA(cudaFuncSetAttribute(mesh_dft_partial_kernel<T, 6, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  TUFRG_CUDA(cudaFuncSetAttribute(mesh_dft_partial_kernel<T, 8, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  TUFRG_CUDA(cudaFuncSetAttribute(mesh_dft_partial_kernel<T, 8, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  TUFRG_CUDA(cudaFuncSetAttribute(bond_dft1_kernel<T, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  TUFRG_CUDA(cudaFuncSetAttribute(bond_dft1_kernel<T, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  cudaError_t e = cudaSuccess;
  for_each_nf([&](auto nf) {
    constexpr int NF = decltype(nf)::value;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(bond_dft2_kernel<T, NF>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mesh_dft_reduce_kernel<T, NF>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mesh_tc_reduce_kernel<NF>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = allow_dynamic_smem(contract_terms_kernel<T, NF>, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(overlap_kernel<T, NF>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  TUFRG_CUDA(e);
  return TUFRG_OK;
}

template <class T>
tufrg_status project_typed(const MultiView& v, const T* y, T* out, void* btv,
                           void* fkv, cudaStream_t st, bool rows) {
  const int kind = rows ? kKindContractRows : kKindContract;
  using V = typename C2<T>::type;
  V* bt = reinterpret_cast<V*>(btv);
  V* fkey = reinterpret_cast<V*>(fkv);
  const bool mesh_tc = sizeof(T) == 4 && v.mesh && v.h[0].mesh_ahi;
  if (v.total(kKindBond) > 0 && mesh_tc) {
    // the quadrature on the tensor cores (the partials in the bt region)
    TUFRG_CHECK(launch_mesh_tc(v.h[0], reinterpret_cast<const float*>(y) +
                                           (rows ? v.h[0].off_wstate : v.h[0].off_state),
                               rows, reinterpret_cast<float*>(bt) + 2 * v.h[0].off_bt, v.d_err,
                               st));
  } else if (v.total(kKindBond) > 0 && v.mesh) {
    const int xt = mesh_xt(v);
    const size_t sm = mesh_partial_smem<T>(xt);
    const int n = v.total(kKindBond);
    const int* pre = v.dprefix(kKindBond);
    if (xt == 6 && rows)
      mesh_dft_partial_kernel<T, 6, true><<<n, 256, sm, st>>>(v.d, pre, v.n, y, bt);
    else if (xt == 6)
      mesh_dft_partial_kernel<T, 6, false><<<n, 256, sm, st>>>(v.d, pre, v.n, y, bt);
    else if (rows)
      mesh_dft_partial_kernel<T, 8, true><<<n, 256, sm, st>>>(v.d, pre, v.n, y, bt);
    else
      mesh_dft_partial_kernel<T, 8, false><<<n, 256, sm, st>>>(v.d, pre, v.n, y, bt);
    TUFRG_CUDA(cudaGetLastError());
  } else if (v.total(kKindBond) > 0) {
    if (rows)
      bond_dft1_kernel<T, true><<<v.total(kKindBond), kDft1Threads, dft1_smem<T>(v), st>>>(
          v.d, v.dprefix(kKindBond), v.n, y, bt);
    else
      bond_dft1_kernel<T, false><<<v.total(kKindBond), kDft1Threads, dft1_smem<T>(v), st>>>(
          v.d, v.dprefix(kKindBond), v.n, y, bt);
    TUFRG_CUDA(cudaGetLastError());
  }
  if (v.total(kKindDft) > 0 && v.mesh) {
    with_nf(v.nf_uniform, [&](auto nf) {
      constexpr int NF = decltype(nf)::value;
      if constexpr (sizeof(T) == 4) {
        if (mesh_tc) {
          mesh_tc_reduce_kernel<NF><<<v.total(kKindDft), 256, mesh_reduce_smem<T>(v), st>>>(
              v.d, v.dprefix(kKindDft), v.n,
              reinterpret_cast<const float*>(bt) + 2 * v.h[0].off_bt, fkey);
          return;
        }
      }
      mesh_dft_reduce_kernel<T, NF><<<v.total(kKindDft), 256, mesh_reduce_smem<T>(v), st>>>(
          v.d, v.dprefix(kKindDft), v.n, bt, fkey);
    });
    TUFRG_CUDA(cudaGetLastError());
  } else if (v.total(kKindDft) > 0) {
    with_nf(v.nf_uniform, [&](auto nf) {
      bond_dft2_kernel<T, decltype(nf)::value><<<v.total(kKindDft), 256, dft2_smem<T>(v), st>>>(
          v.d, v.dprefix(kKindDft), v.n, bt, fkey);
    });
    TUFRG_CUDA(cudaGetLastError());
  }
  if (!v.proj_grouped) {
    with_nf(v.nf_uniform, [&](auto nf) {
      contract_terms_kernel<T, decltype(nf)::value>
          <<<v.total(kind), 256, contract_terms_smem<T>(v), st>>>(
              v.d, v.dprefix(kind), v.n, y, fkey, out, rows ? 1 : 0);
    });
    TUFRG_CUDA(cudaGetLastError());
    return TUFRG_OK;
  }
  if (v.total(kKindOverlap) > 0) {
    with_nf(v.nf_uniform, [&](auto nf) {
      overlap_kernel<T, decltype(nf)::value><<<v.total(kKindOverlap), 256, overlap_smem<T>(v), st>>>(
          v.d, v.dprefix(kKindOverlap), v.n, fkey, bt);
    });
    TUFRG_CUDA(cudaGetLastError());
  }
  with_nf(v.nf_uniform, [&](auto nf) {
    contract_kernel<T, decltype(nf)::value><<<v.total(kind), kCThreads, 0, st>>>(
        v.d, v.dprefix(kind), v.n, y, bt, out, rows ? 1 : 0);
  });
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace

int bond_ctas(int ncx, int nff) {
  return 3 * ncx * ((nff * nff + kDft1Threads - 1) / kDft1Threads);
}

int dft_ctas(int nd) { return 3 * nd * nd; }

size_t fkey_elems(int nd, int nb) { return (size_t)3 * nd * nd * nb * nb; }

int contract_ctas(int nl, int nff, bool grouped) {
  return grouped ? 3 * contract_ctiles(nl, nff) : 3 * ((nl + kTermsL - 1) / kTermsL);
}

size_t bt_region(int ncx, int nd, int nff, int ny_total) {
  return std::max((size_t)3 * ncx * nd * nff * nff, (size_t)ny_total * hstride(nff));
}

int mesh_partial_ctas(int chunks, int nff) { return 3 * chunks * mesh_ab_tiles(nff); }

size_t mesh_partial_elems(int chunks, int nd, int nff) {
  return (size_t)3 * chunks * nd * nd * nff * nff;
}

size_t ctx_bt_elems(const tufrg_ctx* c) {
  const int nd = 2 * c->proj.dmax + 1;
  size_t b = bt_region(c->ncx, nd, c->nff, c->proj.gy_off[3]);
  if (c->mesh) b = std::max(b, mesh_partial_elems(c->mesh_chunks, nd, c->nff));
  // the tensor-core quadrature's FP32 partials [3][kz][mpad][npad] (a complex
  // element holds four of them in FP32 contexts)
  if (c->mesh && c->d_mesh_ahi)
    b = std::max(b, ((size_t)3 * c->mesh_kz * c->mesh_mpad * c->mesh_npad + 3) / 4);
  return b;
}

tufrg_status prepare_project_multi(const MultiView& v) {
  if (v.nff_max > kMaxNf) return TUFRG_ERR_ARG;
  TUFRG_CHECK(prepare_typed<double>(v));
  return prepare_typed<float>(v);
}

tufrg_status launch_project_multi(const MultiView& v, int prec, const void* y, void* out,
                                  void* bt, void* fkey, cudaStream_t st, bool rows) {
  return prec == TUFRG_FP64
             ? project_typed<double>(v, static_cast<const double*>(y), static_cast<double*>(out),
                                     bt, fkey, st, rows)
             : project_typed<float>(v, static_cast<const float*>(y), static_cast<float*>(out), bt,
                                    fkey, st, rows);
}

}  // namespace tufrg
