// Non-uniform meshes, FP32 arithmetic: the quadrature of the key DFT,
//   D_S[m][n] = sum_l A_w[m][l] B_S[n][l],
// with A_w[2x + c][l] the real (c = 0) and imaginary (c = 1) part of
// nl w(l) e^{i l.X_x} (w: mesh_P's weights for S = P, mesh_CD's for C and D;
// scale independent, BF16 hi/lo at setup) and B_S[ab][l] the source
// channel's state entry ab at mesh point l, as a split-K product on the
// tcgen05 tensor cores (BF16 hi/lo operands, three products, FP32
// accumulation in tensor memory).  Per right-hand side:
//   mesh_pack_kernel -- the state transposed to B_S [n][l] (K-major), split
//     into BF16 hi/lo; on the wedge each point's matrix is read from its
//     row's representative through the row's signed permutation;
//   mesh_gemm_kernel -- per (128 position rows, 128 entries, source, split of
//     the points): D partials in FP32, three cp.async stages of 64 points;
// the splits are added in a fixed order by the projection's reduction.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"
#include "tc_util.cuh"

namespace tufrg {
namespace {

using namespace tc;
using bf16 = __nv_bfloat16;

constexpr int kMT = 128;  // rows (positions' parts) per CTA
constexpr int kNT = 128;  // columns (entries) per CTA
constexpr int kKB = 64;   // points per K-block (128 bytes of bf16)
constexpr int kThr = 512;  // 16 warps: warp w reads TMEM lanes 32 (w % 4), columns 32 (w / 4)
constexpr int kStages = 3;

struct MeshTcArgs {
  const bf16 *ahi, *alo;  // [2][mpad][lp] positions' parts x points
  bf16 *bhi, *blo;        // [3][npad][lp] entries x points
  float* part;            // [3][kz][mpad][npad]
  const int2* lrow;       // wedge: (row, g) of each point
  const int* symperm;
  const int* symsign;
  int* err;
  int nl, nff, nrow, lp, mpad, npad, kz, kbs;
};

__device__ __forceinline__ void split_bf16(float v, bf16& hi, bf16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// B_S[n][l] for tiles of 64 points x 32 entries through shared memory: reads
// coalesced along the entries of one point, writes along the points as
// BF16 pairs (two adjacent points per thread).
__global__ void __launch_bounds__(256)
    mesh_pack_kernel(MeshTcArgs a, const float* __restrict__ y, int wedge) {
  __shared__ float tile[64][33];
  const int l0 = blockIdx.x * 64, n0 = blockIdx.y * 32, s = blockIdx.z;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 8 rows of 32
  const int nff2 = a.nff * a.nff;
  for (int r = ty; r < 64; r += 8) {
    const int l = l0 + r, n = n0 + tx;
    float v = 0.f;
    if (l < a.nl && n < nff2) {
      if (wedge) {
        const int2 rg = __ldg(a.lrow + l);
        const int i = n / a.nff, j = n - i * a.nff;
        const int pi = __ldg(a.symperm + rg.y * a.nff + i), pj = __ldg(a.symperm + rg.y * a.nff + j);
        const int sg = __ldg(a.symsign + rg.y * a.nff + i) * __ldg(a.symsign + rg.y * a.nff + j);
        const float w = __ldg(y + ((size_t)s * a.nrow + rg.x) * nff2 + pi * a.nff + pj);
        v = sg > 0 ? w : -w;
      } else {
        v = __ldg(y + ((size_t)s * a.nl + l) * nff2 + n);
      }
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int n = n0 + r, l = l0 + 2 * tx;  // n < npad, l + 1 < lp by the grid
    bf16 h0, g0, h1, g1;
    split_bf16(tile[2 * tx][r], h0, g0);
    split_bf16(tile[2 * tx + 1][r], h1, g1);
    const size_t o = ((size_t)s * a.npad + n) * a.lp + l;
    *reinterpret_cast<__nv_bfloat162*>(a.bhi + o) = __halves2bfloat162(h0, h1);
    *reinterpret_cast<__nv_bfloat162*>(a.blo + o) = __halves2bfloat162(g0, g1);
  }
}

// One CTA: rows [128 bx, +128) x entries [128 by, +128) of source bz / kz,
// points of split bz % kz.  Both operands K-major BF16 hi/lo, loaded by
// cp.async into the 128-byte-swizzled layout; one thread issues the MMAs
// (the two products of A_hi back to back, A_hi kept in the collector).
__global__ void __launch_bounds__(kThr, 1) mesh_gemm_kernel(MeshTcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  constexpr uint32_t kTile = kMT * 128;  // = kNT * 128
  constexpr uint32_t kStage = 4 * kTile;
  const uint32_t ctrl = base + kStages * kStage;  // one mbarrier per stage
  unsigned char* gctrl = gbase + kStages * kStage;
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(gctrl + 32);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gctrl + 36);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = blockIdx.z / a.kz, z = blockIdx.z - s * a.kz;
  const int ws = s == 0 ? 0 : 1;
  const long long m0 = (long long)blockIdx.x * kMT, n0 = (long long)blockIdx.y * kNT;
  const int kb0 = z * a.kbs, nk = min(a.kbs, a.lp / kKB - kb0);
  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) mbar_init(ctrl + 8 * q, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(kNT)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const bf16* Ahi = a.ahi + ((size_t)ws * a.mpad + m0) * a.lp;
  const bf16* Alo = a.alo + ((size_t)ws * a.mpad + m0) * a.lp;
  const bf16* Bhi = a.bhi + ((size_t)s * a.npad + n0) * a.lp;
  const bf16* Blo = a.blo + ((size_t)s * a.npad + n0) * a.lp;

  auto load = [&](int kb, int st_i) {
    const uint32_t st = base + st_i * kStage;
    const long long k0 = (long long)(kb0 + kb) * kKB;
    for (int c = tid; c < 4 * kMT * 8; c += kThr) {
      const int t = c / (kMT * 8), rem = c - t * kMT * 8, row = rem >> 3, ch = rem & 7;
      const bf16* src = (t == 0 ? Ahi : t == 1 ? Alo : t == 2 ? Bhi : Blo) + row * a.lp + k0 + ch * 8;
      cp_async16(st + t * kTile + row * 128 + ((ch ^ (row & 7)) << 4), src);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  // D f32, A and B bf16, both K-major, N = 128, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kNT >> 3) << 17) |
                         ((uint32_t)(kMT >> 4) << 24);
  int last = -1;
  if (nk > 0) load(0, 0);
  if (nk > 1) load(1, 1);
  for (int kb = 0; kb < nk; ++kb) {
    const int st_i = kb % kStages;
    // this K-block's copies (groups up to kb + 1 are committed)
    if (kb + 1 < nk)
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    else
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = base + st_i * kStage;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // 16 points (32 bytes) per instruction
        const uint32_t o = 32u * kk;
        const uint64_t ah = smem_desc(st + o), al = smem_desc(st + kTile + o);
        const uint64_t bh = smem_desc(st + 2 * kTile + o), bl = smem_desc(st + 3 * kTile + o);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n}\n" ::
                "r"(tmem),
            "l"(ah), "l"(bh), "r"(idesc), "r"(acc));
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n}\n" ::
                "r"(tmem),
            "l"(ah), "l"(bl), "r"(idesc), "r"(1u));
        mma_bf16(tmem, al, bh, idesc, 1u);
      }
      mma_commit(ctrl + 8 * st_i);
    }
    last = kb;
    if (kb + 2 < nk) {
      // refill the stage of K-block kb - 1 once its MMAs have completed (the
      // MMAs of kb are queued behind them meanwhile)
      if (kb >= 1 && !mbar_wait(ctrl + 8 * ((kb - 1) % kStages), ((kb - 1) / kStages) & 1)) {
        atomicOr(a.err, 16);
        *abort_flag = 1;
      }
      __syncthreads();
      if (*abort_flag) break;
      load(kb + 2, (kb + 2) % kStages);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (last >= 0 && !mbar_wait(ctrl + 8 * (last % kStages), (last / kStages) & 1)) {
    atomicOr(a.err, 16);
    *abort_flag = 1;
  }
  __syncthreads();  // one decision for the whole CTA (tcgen05.ld is warp-collective)
  const bool ok = !*abort_flag && nk > 0 && last == nk - 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // partials [s][z][mpad][npad]: the thread's row m, 16 entries per load
  constexpr int kCols = kNT / (kThr / 128);  // columns per warp
  const int quad = warp & 3, part = warp >> 2;
  float* out = a.part + (((size_t)s * a.kz + z) * a.mpad + m0 + quad * 32 + lane) * a.npad + n0;
  for (int c0 = part * kCols; c0 < (part + 1) * kCols; c0 += 16) {
    float v[16];
    if (ok) {
      tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = 0.f;  // no points in this split (or a timeout)
    }
#pragma unroll
    for (int j = 0; j < 16; j += 4)
      *reinterpret_cast<float4*>(out + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kNT)
                 : "memory");
  }
}

}  // namespace

size_t mesh_gemm_smem() { return kStages * 4 * (size_t)kMT * 128 + 1024 + 64; }

tufrg_status prepare_mesh_tc() {
  TUFRG_CUDA(cudaFuncSetAttribute(mesh_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)mesh_gemm_smem()));
  return TUFRG_OK;
}

tufrg_status launch_mesh_tc(const PointDesc& d, const float* y, bool wedge, float* part, int* err,
                            cudaStream_t st) {
  MeshTcArgs a;
  a.ahi = static_cast<const bf16*>(d.mesh_ahi);
  a.alo = static_cast<const bf16*>(d.mesh_alo);
  a.bhi = static_cast<bf16*>(d.mesh_bhi);
  a.blo = static_cast<bf16*>(d.mesh_blo);
  a.part = part;
  a.lrow = d.lrow;
  a.symperm = d.symperm;
  a.symsign = d.symsign;
  a.err = err;
  a.nl = d.nl;
  a.nff = d.nff;
  a.nrow = d.nrow;
  a.lp = d.mesh_lp;
  a.mpad = d.mesh_mpad;
  a.npad = d.mesh_npad;
  a.kz = d.mesh_kz;
  a.kbs = d.mesh_kbs;
  const dim3 pg((unsigned)(a.lp / 64), (unsigned)(a.npad / 32), 3);
  mesh_pack_kernel<<<pg, 256, 0, st>>>(a, y, wedge ? 1 : 0);
  TUFRG_CUDA(cudaGetLastError());
  const dim3 gg((unsigned)(a.mpad / kMT), (unsigned)(a.npad / kNT), (unsigned)(3 * a.kz));
  mesh_gemm_kernel<<<gg, kThr, mesh_gemm_smem(), st>>>(a);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace tufrg
