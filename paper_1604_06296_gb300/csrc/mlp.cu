// Learned loop surrogate (not part of the paper's method): a multilayer
// perceptron from (l_x, l_y, ln Lambda, t', mu) to the loops, trained and
// evaluated by the kernels of this file.
//
// Every dense layer is a GEMM D[m][n] = sum_k A[m][k] B[n][k] on the tcgen05
// tensor cores with K-major BF16 hi/lo operand pairs (three products
// A_hi B_hi + A_lo B_hi + A_hi B_lo, as the loop contraction) and an FP32
// accumulator in tensor memory; the epilogue that reads the accumulator out
// applies the layer's operation and writes the operands of the next GEMMs:
//   forward hidden:  z = D + b; store z (FP32) and a = silu(z) as hi/lo
//                    row-major (next layer) and transposed (weight gradient)
//   forward output:  y = D + b (FP32)
//   backward dA:     g = D * silu'(z_prev); store g hi/lo row-major and
//                    transposed; bias gradient by column sums
//   weight gradient: D (FP32), D = G^T A over the batch
// Layer sizes are padded to multiples of 128 (weights and biases zero in the
// padding); batches to multiples of 128 rows whose padded rows get a zero
// loss gradient.  Adam keeps FP32 master weights, moments and the flattened
// gradient; the BF16 hi/lo weight copies (row-major and transposed) are
// regenerated after every update.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "tc_util.cuh"
#include "internal.h"

struct tufrg_surrogate;

namespace tufrg {
namespace {

using namespace tc;
using bf16 = __nv_bfloat16;

constexpr int kGT = 128;          // GEMM threads (4 warps = 128 TMEM lanes)
constexpr int kBM = 128;          // rows per CTA
constexpr int kKB = 64;           // K per K-block (128 bytes of bf16)
constexpr int kMaxLayers = 9;

struct GemmOp {
  const bf16* Ahi;
  const bf16* Alo;
  long long lda;
  const bf16* Bhi;
  const bf16* Blo;
  long long ldb;
  int K;        // multiple of 64
  int* err;
};

__device__ __forceinline__ void split(float v, bf16& hi, bf16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

constexpr int kEmbed = 25;        // fixed features of the five inputs

// The fixed feature map ahead of the first layer: x; cos, sin of k pi x_0
// and k pi x_1 for k = 1..4 (the loops are periodic in l); x_2^2, x_2^3,
// x_2 x_3, x_2 x_4.
__device__ __forceinline__ void embed(const float* x, float* e) {
#pragma unroll
  for (int j = 0; j < 5; ++j) e[j] = x[j];
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    float s0, c0, s1, c1;
    sincospif(k * x[0], &s0, &c0);
    sincospif(k * x[1], &s1, &c1);
    e[1 + 4 * k] = c0;
    e[2 + 4 * k] = s0;
    e[3 + 4 * k] = c1;
    e[4 + 4 * k] = s1;
  }
  e[21] = x[2] * x[2];
  e[22] = x[2] * x[2] * x[2];
  e[23] = x[2] * x[3];
  e[24] = x[2] * x[4];
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// forward hidden layer
struct EpiHidden {
  const float* bias;
  float* Z;
  long long ldz;
  bf16 *Ohi, *Olo;
  long long ldo;
  bf16 *Thi, *Tlo;  // transposed activations (null: not needed)
  long long ldt;
  __device__ void operator()(int m, int n0, const float* v) const {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = n0 + j;
      const float z = v[j] + bias[n];
      Z[m * ldz + n] = z;
      bf16 h, l;
      split(silu(z), h, l);
      Ohi[m * ldo + n] = h;
      Olo[m * ldo + n] = l;
      if (Thi) {
        Thi[n * ldt + m] = h;
        Tlo[n * ldt + m] = l;
      }
    }
  }
};

// forward output layer; with oscale (inference) the standardised outputs
// are mapped back to targets: y scale + shift
struct EpiOut {
  const float* bias;
  float* Y;
  long long ldy;
  const float* oscale;
  const float* oshift;
  __device__ void operator()(int m, int n0, const float* v) const {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = n0 + j;
      float y = v[j] + bias[n];
      if (oscale) y = fmaf(y, oscale[n], oshift[n]);
      Y[m * ldy + n] = y;
    }
  }
};

// backward through the previous layer's activation
struct EpiBwd {
  const float* Z;  // pre-activations of the previous layer
  long long ldz;
  bf16 *Ohi, *Olo;
  long long ldo;
  bf16 *Thi, *Tlo;
  long long ldt;
  float* dbias;  // bias gradient of the previous layer (column sums)
  __device__ void operator()(int m, int n0, const float* v) const {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = n0 + j;
      const float g = v[j] * dsilu(Z[m * ldz + n]);
      bf16 h, l;
      split(g, h, l);
      Ohi[m * ldo + n] = h;
      Olo[m * ldo + n] = l;
      Thi[n * ldt + m] = h;
      Tlo[n * ldt + m] = l;
      float s = g;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) atomicAdd(dbias + n, s);
    }
  }
};

// plain FP32 store (weight gradients)
struct EpiStore {
  float* D;
  long long ldd;
  __device__ void operator()(int m, int n0, const float* v) const {
#pragma unroll
    for (int j = 0; j < 16; ++j) D[m * ldd + n0 + j] = v[j];
  }
};

// One CTA: rows [128 bx, +128) x columns [tn by, +tn) of D, K-blocks of 64
// through two cp.async stages; one thread issues the MMAs.
template <class Epi>
__global__ void __launch_bounds__(kGT, 1) gemm_kernel(GemmOp g, Epi epi, int tn, int tmem_cols) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  const uint32_t a_tile = kBM * 128, b_tile = (uint32_t)tn * 128;
  const uint32_t stage_bytes = 2 * a_tile + 2 * b_tile;
  const uint32_t ctrl = base + 2 * stage_bytes;
  unsigned char* gctrl = gbase + 2 * stage_bytes;
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(gctrl + 16);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gctrl + 20);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long m0 = (long long)blockIdx.x * kBM, n0 = (long long)blockIdx.y * tn;
  if (tid == 0) {
    mbar_init(ctrl, 1);
    mbar_init(ctrl + 8, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int nk = g.K / kKB;

  auto load = [&](int kb, int s) {
    const uint32_t st = base + s * stage_bytes;
    const long long k0 = (long long)kb * kKB;
    for (int c = tid; c < 2 * kBM * 8; c += kGT) {
      const int t = c >= kBM * 8, rem = c - t * kBM * 8, row = rem >> 3, ch = rem & 7;
      cp_async16(st + t * a_tile + row * 128 + ((ch ^ (row & 7)) << 4),
                 (t ? g.Alo : g.Ahi) + (m0 + row) * g.lda + k0 + ch * 8);
    }
    for (int c = tid; c < 2 * tn * 8; c += kGT) {
      const int t = c >= tn * 8, rem = c - t * tn * 8, row = rem >> 3, ch = rem & 7;
      cp_async16(st + 2 * a_tile + t * b_tile + row * 128 + ((ch ^ (row & 7)) << 4),
                 (t ? g.Blo : g.Bhi) + (n0 + row) * g.ldb + k0 + ch * 8);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  // D f32, A and B bf16, both K-major, N = tn, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(tn >> 3) << 17) |
                         ((uint32_t)(kBM >> 4) << 24);
  int last = -1;  // last K-block whose MMAs were committed
  load(0, 0);
  for (int kb = 0; kb < nk; ++kb) {
    const int s = kb & 1;
    if (kb + 1 < nk) {
      // the other stage was read by the MMAs of K-block kb - 1
      if (kb >= 1 && !mbar_wait(ctrl + 8 * ((kb - 1) & 1), ((kb - 1) >> 1) & 1)) {
        atomicOr(g.err, 8);
        *abort_flag = 1;
      }
      __syncthreads();
      if (*abort_flag) break;
      load(kb + 1, (kb + 1) & 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = base + s * stage_bytes;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // 16 k (32 bytes) per instruction
        const uint32_t o = 32u * kk;
        const uint64_t ah = smem_desc(st + o), al = smem_desc(st + a_tile + o);
        const uint64_t bh = smem_desc(st + 2 * a_tile + o);
        const uint64_t bl = smem_desc(st + 2 * a_tile + b_tile + o);
        mma_bf16(tmem, ah, bh, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        mma_bf16(tmem, al, bh, idesc, 1u);
        mma_bf16(tmem, ah, bl, idesc, 1u);
      }
      mma_commit(ctrl + 8 * s);
    }
    last = kb;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // every issued MMA has completed once the last commit has arrived
  if (last >= 0 && !mbar_wait(ctrl + 8 * (last & 1), (last >> 1) & 1)) {
    atomicOr(g.err, 8);
    *abort_flag = 1;
  }
  __syncthreads();  // one decision for the whole CTA (tcgen05.ld is warp-collective)
  const bool ok = !*abort_flag && last == nk - 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = (int)m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < tn; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      epi(row, (int)n0 + c0, v);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

struct LayerTab {
  int n_layers;
  long long off_w[kMaxLayers], off_b[kMaxLayers];
  int k[kMaxLayers], n[kMaxLayers], kp[kMaxLayers], np[kMaxLayers];
  long long n_params;
};

struct WeightPtrs {
  bf16 *Whi[kMaxLayers], *Wlo[kMaxLayers], *WThi[kMaxLayers], *WTlo[kMaxLayers];
  float* b[kMaxLayers];
};

// BF16 hi/lo copies of every layer i (blockIdx.y): W [np][kp] (K-major) and
// W^T [kp][np], and the padded FP32 biases, from the master parameters
__global__ void refresh_kernel(const float* __restrict__ w, LayerTab t, WeightPtrs p) {
  const int i = blockIdx.y;
  const int np = t.np[i], kp = t.kp[i];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < np) p.b[i][e] = e < t.n[i] ? w[t.off_b[i] + e] : 0.f;
  if (e >= np * kp) return;
  const int n = e / kp, k = e % kp;
  const float v = (n < t.n[i] && k < t.k[i]) ? w[t.off_w[i] + (long long)n * t.k[i] + k] : 0.f;
  bf16 h, l;
  split(v, h, l);
  p.Whi[i][e] = h;
  p.Wlo[i][e] = l;
  p.WThi[i][(long long)k * np + n] = h;
  p.WTlo[i][(long long)k * np + n] = l;
}

// Input rows (optionally gathered through idx), embedded, as hi/lo operands
// [mp][64] and transposed [64][mp]; targets gathered to [mp][n_out] FP32.
__global__ void gather_kernel(const float* __restrict__ x, const float* __restrict__ tin,
                              const long long* __restrict__ idx, int count, int mp, int n_out,
                              const float* __restrict__ oshift, const float* __restrict__ oscale,
                              bf16* __restrict__ Xhi, bf16* __restrict__ Xlo,
                              bf16* __restrict__ XThi, bf16* __restrict__ XTlo,
                              float* __restrict__ Tb) {
  const int r = blockIdx.x;
  const bool real = r < count;
  const long long src = real ? (idx ? idx[r] : r) : 0;
  float xin[5], e[kEmbed];
#pragma unroll
  for (int j = 0; j < 5; ++j) xin[j] = real ? x[src * 5 + j] : 0.f;
  embed(xin, e);
  for (int c = threadIdx.x; c < kKB; c += blockDim.x) {
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < kEmbed; ++j)
      if (c == j) v = e[j];
    if (!real) v = 0.f;
    bf16 h, l;
    split(v, h, l);
    Xhi[(long long)r * kKB + c] = h;
    Xlo[(long long)r * kKB + c] = l;
    if (XThi) {
      XThi[(long long)c * mp + r] = h;
      XTlo[(long long)c * mp + r] = l;
    }
  }
  if (Tb)
    for (int c = threadIdx.x; c < n_out; c += blockDim.x)
      Tb[(long long)r * n_out + c] =
          real ? (tin[src * n_out + c] - oshift[c]) / oscale[c] : 0.f;
}

// per-output sums and sums of squares of the targets (FP64), rows split over
// blockIdx.y
__global__ void target_moments_kernel(const float* __restrict__ t, long long n, int n_out,
                                      double* __restrict__ mom) {
  const int c = blockIdx.x;
  double s = 0.0, q = 0.0;
  for (long long r = blockIdx.y * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.y * blockDim.x) {
    const double v = t[r * n_out + c];
    s += v;
    q += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, o);
    q += __shfl_down_sync(0xffffffffu, q, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(mom + 2 * c, s);
    atomicAdd(mom + 2 * c + 1, q);
  }
}

__global__ void target_scaling_kernel(const double* __restrict__ mom, long long n, int n_out,
                                      float* __restrict__ oshift, float* __restrict__ oscale) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_out) return;
  const double mean = mom[2 * c] / n;
  const double var = fmax(mom[2 * c + 1] / n - mean * mean, 0.0);
  oshift[c] = (float)mean;
  oscale[c] = var > 0.0 ? (float)sqrt(var) : 1.f;
}

// dL/dy of L = sum (y - t)^2 / (count n_out) for real rows (zero for padded
// rows and columns) as hi/lo operands, row-major and transposed; the output
// bias gradient (column sums) and the loss.
__global__ void loss_grad_kernel(const float* __restrict__ Y, long long ldy,
                                 const float* __restrict__ Tb, int count, int n_out, int np,
                                 int mp, bf16* __restrict__ Ghi, bf16* __restrict__ Glo,
                                 bf16* __restrict__ GThi, bf16* __restrict__ GTlo,
                                 float* __restrict__ dbias, double* __restrict__ loss) {
  const int r0 = blockIdx.x * kBM;
  const float scale = 2.f / ((float)count * (float)n_out);
  double lsum = 0.0;
  for (int c = threadIdx.x; c < np; c += blockDim.x) {
    float col = 0.f;
    for (int r = r0; r < r0 + kBM; ++r) {
      float d = 0.f;
      if (r < count && c < n_out) {
        const float res = Y[r * ldy + c] - Tb[(long long)r * n_out + c];
        d = scale * res;
        lsum += (double)res * res;
      }
      bf16 h, l;
      split(d, h, l);
      Ghi[(long long)r * np + c] = h;
      Glo[(long long)r * np + c] = l;
      GThi[(long long)c * mp + r] = h;
      GTlo[(long long)c * mp + r] = l;
      col += d;
    }
    atomicAdd(dbias + c, col);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss, s / ((double)count * n_out));
  }
}

// the flattened gradient from the per-layer (padded) weight and bias gradients
__device__ __forceinline__ float grad_at(long long j, const LayerTab& t, float* const* dW,
                                         float* const* db) {
  int i = 0;
  while (i + 1 < t.n_layers && j >= t.off_w[i + 1]) ++i;
  if (j >= t.off_b[i]) return db[i][j - t.off_b[i]];
  const long long e = j - t.off_w[i];
  const int n = (int)(e / t.k[i]), k = (int)(e % t.k[i]);
  return dW[i][(long long)n * t.kp[i] + k];
}

struct GradPtrs {
  float* dW[kMaxLayers];
  float* db[kMaxLayers];
};

__global__ void flatten_grad_kernel(LayerTab t, GradPtrs gp, float* __restrict__ out) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j < t.n_params) out[j] = grad_at(j, t, gp.dW, gp.db);
}

__global__ void adam_kernel(LayerTab t, GradPtrs gp, float* __restrict__ w, float* __restrict__ m,
                            float* __restrict__ v, float lr, float bc1, float bc2) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= t.n_params) return;
  const float g = grad_at(j, t, gp.dW, gp.db);
  const float mj = 0.9f * m[j] + 0.1f * g;
  const float vj = 0.999f * v[j] + 0.001f * g * g;
  m[j] = mj;
  v[j] = vj;
  w[j] -= lr * (mj / bc1) / (sqrtf(vj / bc2) + 1e-8f);
}

// ----------------------------------------------------------- loops <-> rows

struct FeatArgs {
  int ncx, ncy, nl, mp;
  double tp, mu;
  const double* lam;
};

// embedded network inputs of every l of the coarse grid at the scale *lam
// (hi/lo operand rows, padded rows and columns zero)
__global__ void features_kernel(FeatArgs a, bf16* __restrict__ Xhi, bf16* __restrict__ Xlo) {
  const int r = blockIdx.x;
  const double L = a.lam[0];
  float f[5] = {0, 0, 0, 0, 0};
  if (r < a.nl) {
    const int ix = r / a.ncy, iy = r % a.ncy;
    f[0] = (float)(-1.0 + 2.0 * ix / a.ncx);  // l_x / pi
    f[1] = (float)(-1.0 + 2.0 * iy / a.ncy);
    f[2] = (float)((log(L) - log(0.1)) / 4.6);
    f[3] = (float)((a.tp + 0.225) / 0.225);
    f[4] = (float)((a.mu + 0.9) / 0.9);
  }
  float e[kEmbed];
  embed(f, e);
  for (int c = threadIdx.x; c < kKB; c += blockDim.x) {
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < kEmbed; ++j)
      if (c == j) v = e[j];
    if (r >= a.nl) v = 0.f;
    bf16 h, l;
    split(v, h, l);
    Xhi[(long long)r * kKB + c] = h;
    Xlo[(long long)r * kKB + c] = l;
  }
}

// network outputs -> loops [2][nl][nff][nff] (symmetric; forbidden pairs are
// left untouched: the caller's buffer holds zeros there)
__global__ void outputs_to_loops_kernel(const float* __restrict__ Y, long long ldy, int nl,
                                        int npair, const int* __restrict__ pair, int nff,
                                        const double* __restrict__ lam, double* __restrict__ chi) {
  const int l = blockIdx.x;
  const double L = lam[0], inv = 1.0 / (L * (1.0 + L));
  for (int q = threadIdx.x; q < 2 * npair; q += blockDim.x) {
    const int c = q / npair, p = pair[q % npair], m = p / nff, n = p % nff;
    const double v = (double)Y[(long long)l * ldy + q] * inv;
    double* o = chi + ((long long)c * nl + l) * nff * nff;
    o[m * nff + n] = v;
    o[n * nff + m] = v;
  }
}

// training rows of one scale from exact loops
__global__ void loops_to_rows_kernel(const double* __restrict__ chi, int ncx, int ncy, int npair,
                                     const int* __restrict__ pair, int nff, double lam, double tp,
                                     double mu, float* __restrict__ x, float* __restrict__ t) {
  const int l = blockIdx.x, nl = ncx * ncy;
  const int ix = l / ncy, iy = l % ncy;
  if (threadIdx.x == 0) {
    x[l * 5 + 0] = (float)(-1.0 + 2.0 * ix / ncx);
    x[l * 5 + 1] = (float)(-1.0 + 2.0 * iy / ncy);
    x[l * 5 + 2] = (float)((log(lam) - log(0.1)) / 4.6);
    x[l * 5 + 3] = (float)((tp + 0.225) / 0.225);
    x[l * 5 + 4] = (float)((mu + 0.9) / 0.9);
  }
  const double s = lam * (1.0 + lam);
  for (int q = threadIdx.x; q < 2 * npair; q += blockDim.x) {
    const int c = q / npair, p = pair[q % npair];
    t[(long long)l * 2 * npair + q] =
        (float)(s * chi[((long long)c * nl + l) * nff * nff + p]);
  }
}

// relative max-norm error of the surrogate's loops against the exact ones
__global__ void judge_kernel(const double* __restrict__ exact, const double* __restrict__ sur,
                             long long n, unsigned long long* __restrict__ out) {
  unsigned long long dm = 0, em = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    dm = max(dm, (unsigned long long)__double_as_longlong(fabs(exact[i] - sur[i])));
    em = max(em, (unsigned long long)__double_as_longlong(fabs(exact[i])));
  }
  for (int o = 16; o > 0; o >>= 1) {
    dm = max(dm, __shfl_down_sync(0xffffffffu, dm, o));
    em = max(em, __shfl_down_sync(0xffffffffu, em, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, dm);
    atomicMax(out + 1, em);
  }
}

}  // namespace
}  // namespace tufrg

// ------------------------------------------------------------------ host
struct tufrg_surrogate {
  int n_out = 0, width = 0, depth = 0, L = 0;
  tufrg::LayerTab t{};
  float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;  // flat FP32
  int adam_t = 0;
  // per layer
  std::vector<__nv_bfloat16*> Whi, Wlo, WThi, WTlo;
  std::vector<float*> bias, dW, db, Z;
  // activations / gradients for up to mcap rows
  int mcap = 0;
  __nv_bfloat16 *Xhi = nullptr, *Xlo = nullptr, *XThi = nullptr, *XTlo = nullptr;
  std::vector<__nv_bfloat16*> Ahi, Alo, AThi, ATlo, Ghi, Glo, GThi, GTlo;
  float* Y = nullptr;
  float* Tb = nullptr;
  long long* idx = nullptr;
  long long idx_cap = 0;
  double* d_loss = nullptr;
  unsigned long long* d_judge = nullptr;
  int* d_err = nullptr;
  double* chi_judge = nullptr;  // exact loops of a judgement
  size_t chi_judge_elems = 0;
  // output standardisation: the network predicts (target - shift) / scale
  float *oshift = nullptr, *oscale = nullptr;
  bool scaled = false;  // set from the first training set
};

namespace tufrg {
namespace {

template <class T>
bool dalloc(T** p, size_t n) {
  return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) == cudaSuccess;
}

int round_up(int a, int b) { return (a + b - 1) / b * b; }

size_t gemm_smem(int tn) { return 1024 + 2 * (2 * (size_t)kBM * 128 + 2 * (size_t)tn * 128) + 64; }

int tile_n(int N) { return N % 256 == 0 ? 256 : (N % 128 == 0 ? 128 : 64); }

template <class Epi>
tufrg_status gemm(const GemmOp& g, const Epi& epi, int M, int N, cudaStream_t st) {
  if (M % kBM || N % 64 || g.K % kKB || M <= 0 || N <= 0) return TUFRG_ERR_ARG;
  const int tn = tile_n(N);
  const size_t smem = gemm_smem(tn);
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    TUFRG_CUDA(cudaFuncSetAttribute(gemm_kernel<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    smem_optin()));
    attr_set = true;
  }
  int cols = 32;
  while (cols < tn) cols *= 2;
  gemm_kernel<Epi><<<dim3(M / kBM, N / tn), kGT, smem, st>>>(g, epi, tn, cols);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

void free_buffers(tufrg_surrogate* s) {
  std::vector<void*> p = {s->Xhi, s->Xlo, s->XThi, s->XTlo, s->Y, s->Tb};
  for (auto* v : {&s->Ahi, &s->Alo, &s->AThi, &s->ATlo, &s->Ghi, &s->Glo, &s->GThi, &s->GTlo})
    for (auto* q : *v) p.push_back(q);
  for (float* q : s->Z) p.push_back(q);
  for (void* q : p)
    if (q) cudaFree(q);
  s->Xhi = s->Xlo = s->XThi = s->XTlo = nullptr;
  s->Y = s->Tb = nullptr;
  for (auto* v : {&s->Ahi, &s->Alo, &s->AThi, &s->ATlo, &s->Ghi, &s->Glo, &s->GThi, &s->GTlo})
    v->assign(s->L, nullptr);
  s->Z.assign(s->L, nullptr);
  s->mcap = 0;
}

// activation and gradient buffers for mp rows (multiple of 128)
tufrg_status ensure_rows(tufrg_surrogate* s, int mp) {
  if (mp <= s->mcap) return TUFRG_OK;
  free_buffers(s);
  const LayerTab& t = s->t;
  bool ok = dalloc(&s->Xhi, (size_t)mp * kKB) && dalloc(&s->Xlo, (size_t)mp * kKB) &&
            dalloc(&s->XThi, (size_t)mp * kKB) && dalloc(&s->XTlo, (size_t)mp * kKB) &&
            dalloc(&s->Y, (size_t)mp * t.np[s->L - 1]) &&
            dalloc(&s->Tb, (size_t)mp * s->n_out);
  for (int i = 0; ok && i < s->L; ++i) {
    const size_t e = (size_t)mp * t.np[i];
    ok = dalloc(&s->Ghi[i], e) && dalloc(&s->Glo[i], e) && dalloc(&s->GThi[i], e) &&
         dalloc(&s->GTlo[i], e);
    if (ok && i < s->L - 1)
      ok = dalloc(&s->Z[i], e) && dalloc(&s->Ahi[i], e) && dalloc(&s->Alo[i], e) &&
           dalloc(&s->AThi[i], e) && dalloc(&s->ATlo[i], e);
  }
  if (!ok) {
    free_buffers(s);
    return TUFRG_ERR_OOM;
  }
  s->mcap = mp;
  return TUFRG_OK;
}

tufrg_status refresh_weights(tufrg_surrogate* s, cudaStream_t st) {
  const LayerTab& t = s->t;
  WeightPtrs p{};
  int emax = 0;
  for (int i = 0; i < s->L; ++i) {
    p.Whi[i] = s->Whi[i];
    p.Wlo[i] = s->Wlo[i];
    p.WThi[i] = s->WThi[i];
    p.WTlo[i] = s->WTlo[i];
    p.b[i] = s->bias[i];
    emax = std::max(emax, t.np[i] * t.kp[i]);
  }
  refresh_kernel<<<dim3((emax + 255) / 256, s->L), 256, 0, st>>>(s->w, t, p);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

// forward pass of mp rows whose inputs are in Xhi/Xlo; transposed
// activations only when training
tufrg_status forward(tufrg_surrogate* s, int mp, bool train, cudaStream_t st) {
  const LayerTab& t = s->t;
  for (int i = 0; i < s->L; ++i) {
    GemmOp g{};
    g.Ahi = i == 0 ? s->Xhi : s->Ahi[i - 1];
    g.Alo = i == 0 ? s->Xlo : s->Alo[i - 1];
    g.lda = t.kp[i];
    g.Bhi = s->Whi[i];
    g.Blo = s->Wlo[i];
    g.ldb = t.kp[i];
    g.K = t.kp[i];
    g.err = s->d_err;
    if (i < s->L - 1) {
      EpiHidden e{s->bias[i], s->Z[i], t.np[i], s->Ahi[i], s->Alo[i], t.np[i],
                  train ? s->AThi[i] : nullptr, train ? s->ATlo[i] : nullptr, mp};
      TUFRG_CHECK(gemm(g, e, mp, t.np[i], st));
    } else {
      EpiOut e{s->bias[i], s->Y, t.np[i], train ? nullptr : s->oscale,
               train ? nullptr : s->oshift};
      TUFRG_CHECK(gemm(g, e, mp, t.np[i], st));
    }
  }
  return TUFRG_OK;
}

// loss gradient and backward pass (weights' and biases' gradients) of the
// rows gathered in Xhi/XT/Tb by the last forward pass
tufrg_status backward(tufrg_surrogate* s, int count, int mp, cudaStream_t st) {
  const LayerTab& t = s->t;
  const int o = s->L - 1;
  for (int i = 0; i < s->L; ++i)
    TUFRG_CUDA(cudaMemsetAsync(s->db[i], 0, sizeof(float) * t.np[i], st));
  loss_grad_kernel<<<mp / kBM, 128, 0, st>>>(s->Y, t.np[o], s->Tb, count, s->n_out, t.np[o], mp,
                                             s->Ghi[o], s->Glo[o], s->GThi[o], s->GTlo[o],
                                             s->db[o], s->d_loss);
  TUFRG_CUDA(cudaGetLastError());
  for (int i = o; i >= 0; --i) {
    // dW_i [np_i][kp_i] = G_i^T A_{i-1} over the rows
    GemmOp gw{};
    gw.Ahi = s->GThi[i];
    gw.Alo = s->GTlo[i];
    gw.lda = mp;
    gw.Bhi = i == 0 ? s->XThi : s->AThi[i - 1];
    gw.Blo = i == 0 ? s->XTlo : s->ATlo[i - 1];
    gw.ldb = mp;
    gw.K = mp;
    gw.err = s->d_err;
    TUFRG_CHECK(gemm(gw, EpiStore{s->dW[i], t.kp[i]}, t.np[i], t.kp[i], st));
    if (i == 0) break;
    // G_{i-1} = (G_i W_i) * silu'(z_{i-1})
    GemmOp ga{};
    ga.Ahi = s->Ghi[i];
    ga.Alo = s->Glo[i];
    ga.lda = t.np[i];
    ga.Bhi = s->WThi[i];
    ga.Blo = s->WTlo[i];
    ga.ldb = t.np[i];
    ga.K = t.np[i];
    ga.err = s->d_err;
    EpiBwd e{s->Z[i - 1], t.np[i - 1], s->Ghi[i - 1], s->Glo[i - 1], t.np[i - 1],
             s->GThi[i - 1], s->GTlo[i - 1], mp, s->db[i - 1]};
    TUFRG_CHECK(gemm(ga, e, mp, t.kp[i], st));
  }
  return TUFRG_OK;
}

GradPtrs grad_ptrs(tufrg_surrogate* s) {
  GradPtrs g{};
  for (int i = 0; i < s->L; ++i) {
    g.dW[i] = s->dW[i];
    g.db[i] = s->db[i];
  }
  return g;
}

tufrg_status load_rows(tufrg_surrogate* s, const float* x, const float* tin, const long long* idx,
                       int count, int mp, bool transposed, cudaStream_t st) {
  gather_kernel<<<mp, 64, 0, st>>>(x, tin, idx, count, mp, s->n_out, s->oshift, s->oscale,
                                   s->Xhi, s->Xlo,
                                   transposed ? s->XThi : nullptr,
                                   transposed ? s->XTlo : nullptr, tin ? s->Tb : nullptr);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status check_err(tufrg_surrogate* s, cudaStream_t st) {
  int e = 0;
  TUFRG_CUDA(cudaMemcpyAsync(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  if (e) {
    TUFRG_CUDA(cudaMemsetAsync(s->d_err, 0, sizeof(int), st));
    TUFRG_CUDA(cudaStreamSynchronize(st));
    return TUFRG_ERR_TIMEOUT;
  }
  return TUFRG_OK;
}

// seeded 64-bit generator (SplitMix64, Steele, Lea and Flood 2014)
struct SplitMix {
  uint64_t x;
  uint64_t next() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
};

void destroy(tufrg_surrogate* s) {
  cudaDeviceSynchronize();
  free_buffers(s);
  std::vector<void*> p = {s->w,      s->m,       s->v,     s->grad,      s->idx,   s->d_loss,
                          s->d_judge, s->d_err, s->chi_judge, s->oshift, s->oscale};
  for (auto* vec : {&s->Whi, &s->Wlo, &s->WThi, &s->WTlo})
    for (auto* q : *vec) p.push_back(q);
  for (auto* vec : {&s->bias, &s->dW, &s->db})
    for (auto* q : *vec) p.push_back(q);
  for (void* q : p)
    if (q) cudaFree(q);
  delete s;
}

}  // namespace

// ---- pieces the flow uses (declared in internal.h)

tufrg_status surrogate_loops(tufrg_surrogate* s, tufrg_ctx* c, double* chi, cudaStream_t st) {
  const int mp = round_up(c->nl, kBM);
  TUFRG_CHECK(ensure_rows(s, mp));
  FeatArgs a{c->ncx, c->ncy, c->nl, mp, c->p.tp, c->p.mu, c->d_lambda};
  features_kernel<<<mp, 64, 0, st>>>(a, s->Xhi, s->Xlo);
  TUFRG_CUDA(cudaGetLastError());
  TUFRG_CHECK(forward(s, mp, false, st));
  outputs_to_loops_kernel<<<c->nl, 128, 0, st>>>(s->Y, s->t.np[s->L - 1], c->nl, c->npair,
                                                 c->d_pair, c->nff, c->d_lambda, chi);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

// exact loops and the surrogate's at the scale in c->d_lambda: relative
// max-norm error of the surrogate (blocks)
tufrg_status surrogate_judge(tufrg_surrogate* s, tufrg_ctx* c, int exact_prec, double* rel,
                             cudaStream_t st) {
  const size_t n = (size_t)2 * c->nl * c->nff * c->nff;
  if (s->chi_judge_elems < n) {
    if (s->chi_judge) cudaFree(s->chi_judge);
    s->chi_judge = nullptr;
    s->chi_judge_elems = 0;
    if (!dalloc(&s->chi_judge, n)) return TUFRG_ERR_OOM;
    s->chi_judge_elems = n;
  }
  TUFRG_CHECK(launch_loops(c, exact_prec, s->chi_judge, st));  // (clears it first)
  TUFRG_CHECK(surrogate_loops(s, c, c->d_chi, st));
  TUFRG_CUDA(cudaMemsetAsync(s->d_judge, 0, 2 * sizeof(unsigned long long), st));
  judge_kernel<<<152, 256, 0, st>>>(s->chi_judge, c->d_chi, (long long)n, s->d_judge);
  TUFRG_CUDA(cudaGetLastError());
  unsigned long long h[2];
  TUFRG_CUDA(cudaMemcpyAsync(h, s->d_judge, sizeof h, cudaMemcpyDeviceToHost, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  TUFRG_CHECK(check_err(s, st));
  double d, e;
  std::memcpy(&d, &h[0], 8);
  std::memcpy(&e, &h[1], 8);
  *rel = e > 0.0 ? d / e : (d > 0.0 ? INFINITY : 0.0);
  return TUFRG_OK;
}

int surrogate_n_out(const tufrg_surrogate* s) { return s->n_out; }

}  // namespace tufrg

using tufrg::dalloc;

extern "C" {

tufrg_status tufrg_surrogate_create(int32_t n_out, int32_t width, int32_t depth, uint64_t seed,
                                    tufrg_surrogate** out) {
  if (!out) return TUFRG_ERR_ARG;
  *out = nullptr;
  if (n_out < 1 || n_out > 512 || width < 64 || width > 512 || width % 64 || depth < 1 ||
      depth > tufrg::kMaxLayers - 1)
    return TUFRG_ERR_ARG;
  tufrg_surrogate* s = new (std::nothrow) tufrg_surrogate();
  if (!s) return TUFRG_ERR_OOM;
  s->n_out = n_out;
  s->width = width;
  s->depth = depth;
  s->L = depth + 1;
  tufrg::LayerTab& t = s->t;
  t.n_layers = s->L;
  long long off = 0;
  for (int i = 0; i < s->L; ++i) {
    t.k[i] = i == 0 ? tufrg::kEmbed : width;
    t.n[i] = i == s->L - 1 ? n_out : width;
    t.kp[i] = i == 0 ? tufrg::kKB : tufrg::round_up(width, 128);
    t.np[i] = tufrg::round_up(t.n[i], 128);
    t.off_w[i] = off;
    off += (long long)t.n[i] * t.k[i];
    t.off_b[i] = off;
    off += t.n[i];
  }
  t.n_params = off;
  for (auto* v : {&s->Whi, &s->Wlo, &s->WThi, &s->WTlo}) v->assign(s->L, nullptr);
  for (auto* v : {&s->bias, &s->dW, &s->db}) v->assign(s->L, nullptr);
  tufrg::free_buffers(s);
  bool ok = dalloc(&s->w, off) && dalloc(&s->m, off) && dalloc(&s->v, off) &&
            dalloc(&s->grad, off) && dalloc(&s->d_loss, 1) && dalloc(&s->d_judge, 2) &&
            dalloc(&s->d_err, 1) && dalloc(&s->oshift, t.np[s->L - 1]) &&
            dalloc(&s->oscale, t.np[s->L - 1]);
  for (int i = 0; ok && i < s->L; ++i) {
    const size_t e = (size_t)t.np[i] * t.kp[i];
    ok = dalloc(&s->Whi[i], e) && dalloc(&s->Wlo[i], e) && dalloc(&s->WThi[i], e) &&
         dalloc(&s->WTlo[i], e) && dalloc(&s->bias[i], t.np[i]) && dalloc(&s->dW[i], e) &&
         dalloc(&s->db[i], t.np[i]);
  }
  if (!ok) {
    tufrg::destroy(s);
    return TUFRG_ERR_OOM;
  }
  // He-uniform weights, zero biases
  std::vector<float> h(off, 0.f);
  tufrg::SplitMix rng{seed};
  for (int i = 0; i < s->L; ++i) {
    const double a = std::sqrt((i == s->L - 1 ? 3.0 : 6.0) / t.k[i]);
    for (long long j = 0; j < (long long)t.n[i] * t.k[i]; ++j)
      h[t.off_w[i] + j] = (float)(a * (2.0 * rng.uniform() - 1.0));
  }
  tufrg_status st = TUFRG_OK;
  // standardisation over the padded outputs (identity in the padding)
  const int np_out = t.np[s->L - 1];
  const std::vector<float> zero(np_out, 0.f), one(np_out, 1.f);
  if (cudaMemcpy(s->w, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->oshift, zero.data(), sizeof(float) * np_out, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(s->oscale, one.data(), sizeof(float) * np_out, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(s->m, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(s->v, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(s->d_err, 0, sizeof(int)) != cudaSuccess)
    st = TUFRG_ERR_CUDA;
  if (st == TUFRG_OK) st = tufrg::refresh_weights(s, nullptr);
  if (st == TUFRG_OK && cudaDeviceSynchronize() != cudaSuccess) st = TUFRG_ERR_CUDA;
  if (st != TUFRG_OK) {
    tufrg::destroy(s);
    return st;
  }
  *out = s;
  return TUFRG_OK;
}

void tufrg_surrogate_destroy(tufrg_surrogate* s) {
  if (s) tufrg::destroy(s);
}

tufrg_status tufrg_surrogate_n_params(const tufrg_surrogate* s, int64_t* n) {
  if (!s || !n) return TUFRG_ERR_ARG;
  *n = s->t.n_params;
  return TUFRG_OK;
}

tufrg_status tufrg_surrogate_get_params(tufrg_surrogate* s, float* params, void* stream) {
  if (!s || !params) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  TUFRG_CUDA(cudaMemcpyAsync(params, s->w, sizeof(float) * s->t.n_params, cudaMemcpyDeviceToHost,
                             st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

tufrg_status tufrg_surrogate_set_params(tufrg_surrogate* s, const float* params, void* stream) {
  if (!s || !params) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  TUFRG_CUDA(cudaMemcpyAsync(s->w, params, sizeof(float) * s->t.n_params, cudaMemcpyHostToDevice,
                             st));
  TUFRG_CUDA(cudaMemsetAsync(s->m, 0, sizeof(float) * s->t.n_params, st));
  TUFRG_CUDA(cudaMemsetAsync(s->v, 0, sizeof(float) * s->t.n_params, st));
  s->adam_t = 0;
  TUFRG_CHECK(tufrg::refresh_weights(s, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

tufrg_status tufrg_surrogate_get_scaling(tufrg_surrogate* s, float* shift, float* scale,
                                         void* stream) {
  if (!s || !shift || !scale) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  TUFRG_CUDA(cudaMemcpyAsync(shift, s->oshift, sizeof(float) * s->n_out, cudaMemcpyDeviceToHost,
                             st));
  TUFRG_CUDA(cudaMemcpyAsync(scale, s->oscale, sizeof(float) * s->n_out, cudaMemcpyDeviceToHost,
                             st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

tufrg_status tufrg_surrogate_set_scaling(tufrg_surrogate* s, const float* shift,
                                         const float* scale, void* stream) {
  if (!s || (!shift) != (!scale)) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<float> sh(s->n_out, 0.f), sc(s->n_out, 1.f);
  if (shift)
    for (int c = 0; c < s->n_out; ++c) {
      if (!(std::isfinite(scale[c]) && scale[c] > 0.f) || !std::isfinite(shift[c]))
        return TUFRG_ERR_ARG;
      sh[c] = shift[c];
      sc[c] = scale[c];
    }
  TUFRG_CUDA(cudaMemcpyAsync(s->oshift, sh.data(), sizeof(float) * s->n_out,
                             cudaMemcpyHostToDevice, st));
  TUFRG_CUDA(cudaMemcpyAsync(s->oscale, sc.data(), sizeof(float) * s->n_out,
                             cudaMemcpyHostToDevice, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  s->scaled = shift != nullptr;
  return TUFRG_OK;
}

tufrg_status tufrg_surrogate_samples(tufrg_ctx* c, const tufrg_surrogate* s, double lambda,
                                     float* x_dev, float* t_dev, void* stream) {
  if (!c || !s || !x_dev || !t_dev || !(std::isfinite(lambda) && lambda > 0.0) ||
      s->n_out != 2 * c->npair || !c->d_chi)
    return TUFRG_ERR_ARG;
  if (c->mesh) return TUFRG_ERR_STATE;  // the surrogate's inputs are coarse-grid momenta
  cudaStream_t st = (cudaStream_t)stream;
  TUFRG_CHECK(tufrg::launch_set_scalar(c->d_lambda, lambda, st));
  TUFRG_CHECK(tufrg::launch_loops(c, c->p.precision, c->d_chi, st));
  tufrg::loops_to_rows_kernel<<<c->nl, 128, 0, st>>>(c->d_chi, c->ncx, c->ncy, c->npair,
                                                     c->d_pair, c->nff, lambda, c->p.tp, c->p.mu,
                                                     x_dev, t_dev);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status tufrg_surrogate_predict(tufrg_surrogate* s, const float* x_dev, int64_t n,
                                     float* y_dev, void* stream) {
  if (!s || !x_dev || !y_dev || n < 1) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int chunk = 65536;
  for (int64_t r0 = 0; r0 < n; r0 += chunk) {
    const int count = (int)std::min<int64_t>(chunk, n - r0);
    const int mp = tufrg::round_up(count, tufrg::kBM);
    TUFRG_CHECK(tufrg::ensure_rows(s, mp));
    TUFRG_CHECK(tufrg::load_rows(s, x_dev + r0 * 5, nullptr, nullptr, count, mp, false, st));
    TUFRG_CHECK(tufrg::forward(s, mp, false, st));
    TUFRG_CUDA(cudaMemcpy2DAsync(y_dev + r0 * s->n_out, sizeof(float) * s->n_out, s->Y,
                                 sizeof(float) * s->t.np[s->L - 1], sizeof(float) * s->n_out,
                                 count, cudaMemcpyDeviceToDevice, st));
  }
  return TUFRG_OK;
}

tufrg_status tufrg_surrogate_loss_grad(tufrg_surrogate* s, const float* x_dev,
                                       const float* t_dev, int64_t n, double* loss, float* grad,
                                       void* stream) {
  if (!s || !x_dev || !t_dev || n < 1 || n > 65536 || !loss) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int count = (int)n, mp = tufrg::round_up(count, tufrg::kBM);
  TUFRG_CHECK(tufrg::ensure_rows(s, mp));
  TUFRG_CUDA(cudaMemsetAsync(s->d_loss, 0, sizeof(double), st));
  TUFRG_CHECK(tufrg::load_rows(s, x_dev, t_dev, nullptr, count, mp, true, st));
  TUFRG_CHECK(tufrg::forward(s, mp, true, st));
  TUFRG_CHECK(tufrg::backward(s, count, mp, st));
  const long long np = s->t.n_params;
  tufrg::flatten_grad_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(
      s->t, tufrg::grad_ptrs(s), s->grad);
  TUFRG_CUDA(cudaGetLastError());
  TUFRG_CUDA(cudaMemcpyAsync(loss, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (grad)
    TUFRG_CUDA(cudaMemcpyAsync(grad, s->grad, sizeof(float) * np, cudaMemcpyDeviceToHost, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return tufrg::check_err(s, st);
}

tufrg_status tufrg_surrogate_train(tufrg_surrogate* s, const float* x_dev, const float* t_dev,
                                   int64_t n, int32_t epochs, int32_t batch, double lr,
                                   uint64_t seed, double* loss_hist, void* stream) {
  if (!s || !x_dev || !t_dev || n < 1 || epochs < 1 || batch < 1 || batch > 65536 ||
      !(lr > 0.0))
    return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int mpb = tufrg::round_up(batch, tufrg::kBM);
  TUFRG_CHECK(tufrg::ensure_rows(s, mpb));
  if (s->idx_cap < n) {
    if (s->idx) cudaFree(s->idx);
    s->idx = nullptr;
    s->idx_cap = 0;
    if (!dalloc(&s->idx, (size_t)n)) return TUFRG_ERR_OOM;
    s->idx_cap = n;
  }
  if (!s->scaled) {  // standardise the outputs with the moments of this training set
    double* mom = nullptr;
    if (!dalloc(&mom, 2 * (size_t)s->n_out)) return TUFRG_ERR_OOM;
    cudaMemsetAsync(mom, 0, sizeof(double) * 2 * s->n_out, st);
    tufrg::target_moments_kernel<<<dim3(s->n_out, 64), 256, 0, st>>>(t_dev, n, s->n_out, mom);
    tufrg::target_scaling_kernel<<<(s->n_out + 127) / 128, 128, 0, st>>>(mom, n, s->n_out,
                                                                          s->oshift, s->oscale);
    const cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(mom);
    TUFRG_CUDA(e);
    s->scaled = true;
  }
  std::vector<long long> perm(n);
  tufrg::SplitMix rng{seed};
  const long long steps_per_epoch = (n + batch - 1) / batch;
  const long long total = steps_per_epoch * epochs;
  const long long np = s->t.n_params;
  long long step = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (long long i = 0; i < n; ++i) perm[i] = i;
    for (long long i = n - 1; i > 0; --i) std::swap(perm[i], perm[rng.next() % (uint64_t)(i + 1)]);
    TUFRG_CUDA(cudaMemcpyAsync(s->idx, perm.data(), sizeof(long long) * n, cudaMemcpyHostToDevice,
                               st));
    TUFRG_CUDA(cudaMemsetAsync(s->d_loss, 0, sizeof(double), st));
    for (long long b0 = 0; b0 < n; b0 += batch, ++step) {
      const int count = (int)std::min<long long>(batch, n - b0);
      const int mp = tufrg::round_up(count, tufrg::kBM);
      TUFRG_CHECK(tufrg::load_rows(s, x_dev, t_dev, s->idx + b0, count, mp, true, st));
      TUFRG_CHECK(tufrg::forward(s, mp, true, st));
      TUFRG_CHECK(tufrg::backward(s, count, mp, st));
      ++s->adam_t;
      const double frac = (double)step / (double)std::max(1LL, total - 1);
      const double lr_t = lr * (0.01 + 0.99 * 0.5 * (1.0 + std::cos(M_PI * frac)));
      const float bc1 = (float)(1.0 - std::pow(0.9, s->adam_t));
      const float bc2 = (float)(1.0 - std::pow(0.999, s->adam_t));
      tufrg::adam_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(
          s->t, tufrg::grad_ptrs(s), s->w, s->m, s->v, (float)lr_t, bc1, bc2);
      TUFRG_CUDA(cudaGetLastError());
      TUFRG_CHECK(tufrg::refresh_weights(s, st));
    }
    double l = 0.0;
    TUFRG_CUDA(cudaMemcpyAsync(&l, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    TUFRG_CUDA(cudaStreamSynchronize(st));  // also keeps perm alive for the copy
    if (loss_hist) loss_hist[ep] = l / (double)steps_per_epoch;
    TUFRG_CHECK(tufrg::check_err(s, st));
  }
  return TUFRG_OK;
}

tufrg_status tufrg_surrogate_attach(tufrg_ctx* c, tufrg_surrogate* s, int32_t judge_every,
                                    double tol) {
  if (!c) return TUFRG_ERR_ARG;
  if (!s) {
    c->sur = nullptr;
    return TUFRG_OK;
  }
  if (s->n_out != 2 * c->npair || judge_every < 1 || !(tol > 0.0) || !c->d_chi)
    return TUFRG_ERR_ARG;
  if (c->mesh) return TUFRG_ERR_STATE;
  c->sur = s;
  c->sur_every = judge_every;
  c->sur_tol = tol;
  tufrg::flow_drop_graphs(c);
  return TUFRG_OK;
}

}  // extern "C"
