// Step ii (Eq. chis) on the 5th-generation tensor cores (tcgen05, TMEM, TMA).
//
//   chi_dot_{pair}(l) = sum_k F_{pair}(k) W(k, l)
//
// as D[row = l-representative][n = pair] = sum_k W[row][k] F[n][k] with the
// operands split into high and low parts of a narrow type (BF16x3:
// bf16 hi/lo, kind::f16; 3xTF32: tf32 hi/lo, kind::tf32) and three products
// W_hi F_hi + W_lo F_hi + W_hi F_lo accumulated in FP32 in tensor memory;
// the split-K partial sums of each CTA are combined (fixed order, compensated
// FP32 pairs, FP64 result) by a second kernel.  The propagator operand W is
// generated in registers from the per-scale FP32 table (alpha = Omega /
// (Omega + |xi|) and xi, extended by a wrap-around halo so p +- l/2 is one
// add from p) with
// the same closed-form frequency integral as the FP64 path, and written
// straight into the 128B-swizzled K-major shared-memory layout the MMA reads;
// F (scale independent) arrives by TMA (one 2-D box per K-block and part).
// Both channels share W's table reads and divisions and have their own
// accumulator.
//
// Persistent CTAs (one per SM, 17 warps) take work items -- (point, tile of
// up to 128 l-rows, range of K-blocks) of any number of points -- from a
// queue ordered by cost.  The rows of a point are spread evenly over its
// tiles.  Warps 0-15 produce the W tiles of a K-block (8 rows each, lanes
// along k, table loads of several rows in flight; one thread of warp 0 also
// starts the F copies), then read the accumulators out (warp w reads the 32
// TMEM lanes 32 (w % 4).. of channel (w / 4) % 2, half of the columns).
// Warp 16 owns TMEM and one of its threads issues the MMAs.  Two pipeline
// stages, mbarriers full (producers), tma (F bytes) and empty (MMAs done),
// whose phases run on across items; every wait is bounded in time and a
// timeout sets an error word, stops the pipeline, waits for the copies in
// flight, drains the issued MMAs and frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "device_util.cuh"
#include "tc_util.cuh"

namespace tufrg {
namespace {

using namespace tc;

constexpr int kRows = 128;          // MMA M: l-representatives per CTA
constexpr int kProducers = 16;      // producer warps
constexpr int kThreads = 32 * (kProducers + 1);
constexpr int kRowBytes = 128;      // one 128B-swizzle row per K-block
constexpr int kWTile = kRows * kRowBytes;  // 16 KB
constexpr int kDepth = 3;           // producer units in flight (table gathers ahead)

template <int PREC>
struct Prec;
template <>
struct Prec<TUFRG_BF16X3> {
  static constexpr int kElem = 2;      // bytes
  static constexpr int kPerLane = 2;   // k per lane per row
  static constexpr uint32_t kFormat = 1;  // BF16
  struct Buf {
    float4 v[2];  // table pairs at p + l/2, p - l/2
  };
};
template <>
struct Prec<TUFRG_3XTF32> {
  static constexpr int kElem = 4;
  static constexpr int kPerLane = 1;
  static constexpr uint32_t kFormat = 2;  // TF32
  struct Buf {
    float2 v[4];  // table entries at p +- l/2 of two rows
  };
};

// CU: use of the A-operand collector buffer -- 0: none, 1: fill (A read from
// shared memory and kept), 2: lastuse (A from the collector, then released)
template <int PREC, int CU = 0>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
#define TUFRG_MMA(KIND, COLL)                                                          \
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"                          \
               " tcgen05.mma.cta_group::1.kind::" KIND COLL " [%0], %1, %2, %3, p;\n}\n" \
               ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc))
  if constexpr (PREC == TUFRG_BF16X3) {
    if constexpr (CU == 1) TUFRG_MMA("f16", ".collector::a::fill");
    else if constexpr (CU == 2) TUFRG_MMA("f16", ".collector::a::lastuse");
    else TUFRG_MMA("f16", "");
  } else {
    if constexpr (CU == 1) TUFRG_MMA("tf32", ".collector::a::fill");
    else if constexpr (CU == 2) TUFRG_MMA("tf32", ".collector::a::lastuse");
    else TUFRG_MMA("tf32", "");
  }
#undef TUFRG_MMA
}

// approximate reciprocal (PTX rcp.approx: relative error below 2^-22)
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Closed-form frequency integral of the two loops for two propagator pairs
// at once, from the table values alpha = Omega A = Omega / (Omega + |xi|)
// and the signed xi of both propagators (a at p + l/2, b at p - l/2).  With
// h(x) = x (Omega + 3x) / (Omega + x)^3 (so that J = -sgn(xi) h(|xi|) / 4)
// the weights are, times Omega^2 (the factor 1/Omega^2 is applied in the
// combination of the partial sums, with the -1/4 and +1/4):
//   Omega^2 D = Omega^2 h[|xi_a|, |xi_b|]
//     = a_a a_b (5 (a_a + a_b) - 3 - 2 (a_a^2 + a_a a_b + a_b^2)),  a = alpha,
//   Omega^2 S = Omega^2 (h_a + h_b) / (|xi_a| + |xi_b|)
//     = (xi_a a_a^2 (3 - 2 a_a) + xi_b' a_b^2 (3 - 2 a_b)) / (xi_a + xi_b'),
// from Omega^2 h(x) = x a^2 (3 - 2a) (Omega + 3x = (3 - 2a) (Omega + x)) and
// xi_b' = xi_b carried over to the sign of xi_a: numerator and denominator
// of S are sums of two terms of one sign, 3 - 2a lies in [1, 3), and the
// constants are plain numbers.  The particle-particle weight is S for
// propagators of one sign, D else, and the particle-hole weight the other
// one.  The table holds |xi| no smaller than 1e-30 (sign kept): at xi_a =
// xi_b = 0 both are 1, the common limit.
__device__ __forceinline__ void weights(const float2 aa, const float2 xa, const float2 ab,
                                        const float2 xb, float2& wpp, float2& wph) {
  const float2 sa = add2(aa, ab), pa = mul2(aa, ab);
  const float2 q = fma2(sa, make_float2(-2.f, -2.f), make_float2(5.f, 5.f));
  const float2 r = fma2(sa, q, make_float2(-3.f, -3.f));  // -3 + 5 sa - 2 sa^2
  const float2 D = mul2(pa, fma2(pa, make_float2(2.f, 2.f), r));
  const float2 va = mul2(aa, fma2(aa, make_float2(-2.f, -2.f), make_float2(3.f, 3.f)));
  const float2 vb = mul2(ab, fma2(ab, make_float2(-2.f, -2.f), make_float2(3.f, 3.f)));
  const float2 xs = make_float2(copysignf(xb.x, xa.x), copysignf(xb.y, xa.y));
  const float2 num = fma2(mul2(xa, aa), va, mul2(mul2(xs, ab), vb));
  const float2 den = add2(xa, xs);
  const float2 S = mul2(num, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
  const float2 sg = mul2(xa, xb);
  const bool s0 = sg.x > 0.f, s1 = sg.y > 0.f;
  wpp = make_float2(s0 ? S.x : D.x, s1 ? S.y : D.y);
  wph = make_float2(s0 ? D.x : S.x, s1 ? D.y : S.y);
}

// bf16x2 high parts (round to nearest) and low parts (the remainders,
// rounded) of two floats
__device__ __forceinline__ void split_bf16(float2 w, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __float22bfloat162_rn(w);
  const __nv_bfloat162 l = __float22bfloat162_rn(sub2(w, __bfloat1622float2(h)));
  std::memcpy(&hi, &h, 4);
  std::memcpy(&lo, &l, 4);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

struct TcArgs {
  const PointDesc* pts;
  const int4* items;  // (point, l-tile, first K-block, K-blocks), costliest first
  int n_items;
  int* counter;       // items claimed after the first gridDim.x (zero before the launch)
  float* partial;     // per point [ksplit][2][npad][nrow_pad] at off_partial
  int* err;
  int kbps;           // K-blocks per full item: split = first K-block / kbps
  int npad_max, tmem_cols;
};

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) loops_tc_kernel(TcArgs a) {
  using P = Prec<PREC>;
  constexpr int KB = kRowBytes / P::kElem;  // k per K-block
  // producer pipeline unit: one row at two loop points (BF16) or two rows at
  // one loop point (TF32) -- four table entries, one paired weight evaluation
  constexpr int kUnitRows = P::kPerLane == 2 ? 1 : 2;
  constexpr int kUnits = kRows / kProducers / kUnitRows;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  const uint32_t fmax = (uint32_t)a.npad_max * kRowBytes;
  const uint32_t stage_bytes = 4u * kWTile + 2u * fmax;
  // per stage: W pp_hi, pp_lo, ph_hi, ph_lo, F hi, F lo
  const uint32_t ctrl = base + 2u * stage_bytes;
  const uint32_t bar_full = ctrl, bar_tma = ctrl + 16, bar_empty = ctrl + 32,
                 bar_done = ctrl + 48;
  unsigned char* gctrl = gbase + 2u * stage_bytes;
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(gctrl + 56);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gctrl + 60);
  volatile int4* s_item = reinterpret_cast<volatile int4*>(gctrl + 64);
  int* s_off = reinterpret_cast<int*>(gctrl + 128);     // 3xTF32: row offsets
  int2* s_idx = reinterpret_cast<int2*>(gctrl + 128);   // BF16X3: row gather indices

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(bar_full + 8 * s, kProducers);
      mbar_init(bar_tma + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kProducers) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // this producer lane writes bytes [col, col + 4) of rows r = warp + 16 i;
  // all its rows have r % 8 == warp % 8, so the swizzled offset is fixed
  const uint32_t col = (uint32_t)(P::kPerLane * lane) * P::kElem;
  const uint32_t swz = (((col >> 4) ^ (uint32_t)(warp & 7)) << 4) | (col & 15);

  uint32_t g = 0;  // K-blocks this CTA has put through the pipeline
  uint32_t j = 0;  // items this CTA has finished (phase of bar_done)
  int tma_last = -1;  // warp 0, lane 0: last K-block (count g) whose F it requested
  // thread 0: the CTA's next item -- its own index first (the launch has at
  // most one CTA per item), then claimed from the counter during the current
  // item's last K-blocks, so that the claim's round trip overlaps them
  // (-1: claim at the top of the loop)
  int next_it = blockIdx.x;
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = next_it >= 0 ? next_it : (int)gridDim.x + atomicAdd(a.counter, 1);
      next_it = -1;
      const int4 v = it < a.n_items ? a.items[it] : make_int4(-1, 0, 0, 0);
      s_item->x = v.x;
      s_item->y = v.y;
      s_item->z = v.z;
      s_item->w = v.w;
    }
    __syncthreads();
    const int pt = s_item->x, tile = s_item->y, kb0 = s_item->z, cnt = s_item->w;
    if (pt < 0 || *abort_flag) break;
    const PointDesc& pd = a.pts[pt];
    if (pd.skip && *pd.skip) {  // finished point: nothing to do
      __syncthreads();
      continue;
    }
    // rows [row0, row0 + nvalid) of the point: the rows [row_lo, row_hi) the
    // view computes spread evenly over their tiles (at most 128 each)
    const int nr = pd.row_hi - pd.row_lo, tiles = (nr + kRows - 1) / kRows;
    const int row0 = pd.row_lo + (tile * nr) / tiles;
    const int nvalid = pd.row_lo + ((tile + 1) * nr) / tiles - row0;
    if constexpr (P::kPerLane == 2) {
      // every lane's first loop point has the parity pib of the first loop
      // point (neighbour pairs iy, iy + 1 with iy even, even row width), so
      // the pair of p + l/2 is entry (pb >> 1) + a of the even or odd pair
      // array, with a fixed per row: (idx_a, idx_b) into [even | odd] for
      // p + l/2 and p - l/2
      const int pib = pd.kbase[0] & 1, half = (pd.n_ext + 1) / 2;
      for (int r = threadIdx.x; r < kRows; r += kThreads) {
        const int off = r < nvalid ? pd.rowoff[row0 + r] : 0;
        const int qa = pib + off, qb = pib - off;  // of one parity
        const int odd = (qa & 1) * half;
        s_idx[r] = make_int2((qa >> 1) + odd, (qb >> 1) + odd);
      }
    } else {
      for (int r = threadIdx.x; r < kRows; r += kThreads)
        s_off[r] = r < nvalid ? pd.rowoff[row0 + r] : 0;
    }
    __syncthreads();
    const int npad = pd.npad, nsets = pd.nsets;

    if (warp < kProducers) {
      // ---------------------------------------------------------- producers
      // BF16X3: pairs (alpha_q, alpha_q+1, xi_q, xi_q+1) of even q at ext, of
      // odd q at ext + (n_ext + 1) / 2, read at the row's s_idx; 3xTF32:
      // (alpha_q, xi_q) per point
      const float4* ext = pd.ext;
      const float2* ext2 = reinterpret_cast<const float2*>(pd.ext);
      const uint32_t fbytes = (uint32_t)npad * kRowBytes;  // one F part per K-block
      // The table gathers run kDepth - 1 units ahead of the arithmetic, in a
      // ring of register buffers, across K-block boundaries too (the gathers
      // of the next K-block's first units are issued while the last units of
      // this one are computed).  Every warp gathers and computes the same
      // number of units per K-block, without a branch per unit (the compiler
      // interleaves the units): rows without an l (fewer than 16 per tile)
      // read offset 0 and their accumulator rows are never read.
      using Buf = typename P::Buf;
      auto load_unit = [&](int u, int pb, Buf& b) {
        if constexpr (P::kPerLane == 2) {  // one row, two loop points: one pair each side
          const int2 ix = s_idx[warp + kProducers * u];
          const float4* lb = ext + (pb >> 1);
          b.v[0] = __ldg(lb + ix.x);
          b.v[1] = __ldg(lb + ix.y);
        } else {  // two rows, one loop point
          const int off0 = s_off[warp + kProducers * (2 * u)];
          const int off1 = s_off[warp + kProducers * (2 * u + 1)];
          b.v[0] = __ldg(ext2 + (pb + off0));
          b.v[1] = __ldg(ext2 + (pb - off0));
          b.v[2] = __ldg(ext2 + (pb + off1));
          b.v[3] = __ldg(ext2 + (pb - off1));
        }
      };
      auto do_unit = [&](int u, unsigned char* stg, const Buf& b) {
        float2 wpp, wph;
        if constexpr (P::kPerLane == 2)
          weights(make_float2(b.v[0].x, b.v[0].y), make_float2(b.v[0].z, b.v[0].w),
                  make_float2(b.v[1].x, b.v[1].y), make_float2(b.v[1].z, b.v[1].w), wpp, wph);
        else
          weights(make_float2(b.v[0].x, b.v[2].x), make_float2(b.v[0].y, b.v[2].y),
                  make_float2(b.v[1].x, b.v[3].x), make_float2(b.v[1].y, b.v[3].y), wpp, wph);
        if constexpr (PREC == TUFRG_BF16X3) {
          uint32_t v[4];
          split_bf16(wpp, v[0], v[1]);
          split_bf16(wph, v[2], v[3]);
          // plain stores (the compiler may interleave the units around them);
          // the proxy fence before the stage's arrive orders them for the MMA
          unsigned char* dst = stg + (warp + kProducers * u) * kRowBytes + swz;
#pragma unroll
          for (int t = 0; t < 4; ++t) *reinterpret_cast<uint32_t*>(dst + t * kWTile) = v[t];
        } else {
          const float w[2][2] = {{wpp.x, wph.x}, {wpp.y, wph.y}};
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            uint32_t v[4];
            v[0] = tf32_rna(w[r][0]);
            v[1] = tf32_rna(w[r][0] - __uint_as_float(v[0]));
            v[2] = tf32_rna(w[r][1]);
            v[3] = tf32_rna(w[r][1] - __uint_as_float(v[2]));
            unsigned char* dst = stg + (warp + kProducers * (2 * u + r)) * kRowBytes + swz;
#pragma unroll
            for (int t = 0; t < 4; ++t) *reinterpret_cast<uint32_t*>(dst + t * kWTile) = v[t];
          }
        }
      };
      // The K-blocks of the item with NU units per warp (rows warp + 16 u, u <
      // NU: the tile's rows need ceil(nvalid / 16) of the kUnits, BF16X3).
      // Unit u uses ring slot u % kDepth; when NU is not a multiple of
      // kDepth the slots of the next K-block's first units are moved to 0..
      // after each K-block (register moves instead of a second copy of the
      // code per ring phase).
      auto produce = [&](auto nu) {
        constexpr int NU = decltype(nu)::value;
        Buf buf[kDepth];
        // this lane's first loop point of a K-block as an offset into the halo
        // table (padding points use a valid entry: their F is zero); BF16X3
        // lanes take loop points 2 lane, 2 lane + 1 of the K-block, neighbours
        // iy, iy + 1 of one column, i.e. table entries pb, pb + 1
        int pb = cnt > 0 ? __ldg(pd.kbase + kb0 * KB + P::kPerLane * lane) : 0;
#pragma unroll
        for (int t = 0; t < kDepth - 1; ++t)
          if (cnt > 0 && t < NU) load_unit(t, pb, buf[t]);
        for (int kb = 0; kb < cnt; ++kb) {
          const uint32_t gk = g + kb;
          const uint32_t s = gk & 1;
          if (gk >= 2 && !mbar_wait_sleep(bar_empty + 8 * s, ((gk >> 1) + 1) & 1)) {
            atomicOr(a.err, 1);
            *abort_flag = 1;
          }
          if (*abort_flag) break;
          const uint32_t st = base + s * stage_bytes;
          const int k0 = (kb0 + kb) * KB;
          if (warp == 0 && lane == 0) {  // F of this K-block, both parts, by TMA
            mbar_arrive_expect_tx(bar_tma + 8 * s, 2u * fbytes);
            tma_load_2d(st + 4u * kWTile, pd.tmap, k0, 0, bar_tma + 8 * s);
            tma_load_2d(st + 4u * kWTile + fmax,
                        static_cast<const unsigned char*>(pd.tmap) + 128, k0, 0,
                        bar_tma + 8 * s);
            tma_last = (int)gk;
            if (kb == (cnt > 2 ? cnt - 2 : 0)) next_it = (int)gridDim.x + atomicAdd(a.counter, 1);
          }
          unsigned char* stg = gbase + (st - base);
          // (after the item's last K-block the ring gathers this one's first
          // units again: valid addresses, no branch)
          const int pbn = kb + 1 < cnt ? __ldg(pd.kbase + k0 + KB + P::kPerLane * lane) : pb;
#pragma unroll
          for (int u = 0; u < NU; ++u) {
            const int t = u + kDepth - 1;  // unit gathered now, into the slot unit u - 1 freed
            if (t < NU)
              load_unit(t, pb, buf[t % kDepth]);
            else if (t - NU < NU)
              load_unit(t - NU, pbn, buf[t % kDepth]);
            do_unit(u, stg, buf[u % kDepth]);
          }
          if constexpr (NU % kDepth != 0) {
            Buf nxt[kDepth - 1];
#pragma unroll
            for (int j = 0; j < kDepth - 1; ++j) nxt[j] = buf[(NU + j) % kDepth];
#pragma unroll
            for (int j = 0; j < kDepth - 1; ++j) buf[j] = nxt[j];
          }
          pb = pbn;
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar_full + 8 * s);
        }
      };
      if constexpr (P::kPerLane == 2) {
        const int need = (nvalid + kProducers - 1) / kProducers;  // units of this tile
        if (need <= 4)
          produce(std::integral_constant<int, 4>{});
        else if (need == 5)
          produce(std::integral_constant<int, 5>{});
        else if (need == 6)
          produce(std::integral_constant<int, 6>{});
        else if (need == 7)
          produce(std::integral_constant<int, 7>{});
        else
          produce(std::integral_constant<int, kUnits>{});
      } else {
        produce(std::integral_constant<int, kUnits>{});
      }
    } else if (lane == 0) {
      // ------------------------------------------------------- MMA issuer
      // K-blocks go round-robin to nsets accumulator sets (shorter FP32
      // accumulation chains); set q, channel c at TMEM columns (2 q + c) npad
      const uint32_t idesc = (1u << 4) | (P::kFormat << 7) | (P::kFormat << 10) |
                             ((uint32_t)(npad >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
      for (int kb = 0; kb < cnt; ++kb) {
        const uint32_t gk = g + kb;
        const uint32_t s = gk & 1;
        if (!mbar_wait_sleep(bar_full + 8 * s, (gk >> 1) & 1) ||
            !mbar_wait_sleep(bar_tma + 8 * s, (gk >> 1) & 1)) {
          atomicOr(a.err, 2);
          *abort_flag = 1;
        }
        if (*abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = base + s * stage_bytes;
        const uint32_t fh = st + 4u * kWTile, fl = fh + fmax;
        const int set = kb % nsets;
        const bool first = kb < nsets;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of K per instruction
          const uint32_t o = 32u * kk;
          const uint64_t bh = smem_desc(fh + o), bl = smem_desc(fl + o);
#pragma unroll
          for (int ch = 0; ch < 2; ++ch) {
            const uint32_t d = tmem + (uint32_t)((2 * set + ch) * npad);
            const uint64_t ah = smem_desc(st + (2 * ch) * kWTile + o);
            const uint64_t al = smem_desc(st + (2 * ch + 1) * kWTile + o);
            // the two products of W_hi in a row: the second takes W_hi from
            // the tensor core's A collector instead of shared memory
            mma<PREC, 1>(d, ah, bh, idesc, !(first && kk == 0));
            mma<PREC, 2>(d, ah, bl, idesc, 1);
            mma<PREC>(d, al, bh, idesc, 1);
          }
        }
        mma_commit(bar_empty + 8 * s);
      }
      mma_commit(bar_done);  // arrives once every issued MMA has completed
    }

    // ----------------------------------------------------------- epilogue
    if (warp < kProducers) {
      // all producer warps: warp w reads TMEM lanes 32 (w % 4).. of channel
      // (w / 4) % 2, the 16-column blocks w / 8, w / 8 + 2, ...
      const bool ok = mbar_wait_sleep(bar_done, j & 1);
      if (!ok) {
        atomicOr(a.err, 4);
        *abort_flag = 1;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ok && !*abort_flag) {
        const int quad = warp & 3, ch = (warp >> 2) & 1, half = warp >> 3;
        const int row = quad * 32 + lane;
        const int sets = min(nsets, cnt);
        const int split = kb0 / a.kbps;
        float* out = a.partial + pd.off_partial +
                     (size_t)(split * 2 + ch) * npad * pd.nrow_pad + row0 + row;
        for (int c0 = 16 * half; c0 < npad; c0 += 32) {
          float acc[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) acc[q] = 0.f;
          for (int q = 0; q < sets; ++q) {
            uint32_t r[16];
            const uint32_t taddr =
                tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)((2 * q + ch) * npad + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, "
                "%9, %10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[e] += __uint_as_float(r[e]);
          }
          if (row < nvalid) {  // the next tile's rows follow directly
#pragma unroll
            for (int e = 0; e < 16; ++e) out[(size_t)(c0 + e) * pd.nrow_pad] = acc[e];
          }
        }
      }
    }
    g += cnt;
    ++j;
    // the accumulators are read and s_off, s_item are free for the next item
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // after a timeout: the F copies this CTA started land before it exits
  if (threadIdx.x == 0 && tma_last >= 0 && *abort_flag) {
    const uint32_t gk = (uint32_t)tma_last;
    if (!mbar_wait(bar_tma + 8 * (gk & 1), (gk >> 1) & 1)) atomicOr(a.err, 8);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kProducers) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols)
                 : "memory");
  }
}

constexpr int kTableBlock = 256;

// Per-scale FP32 table (alpha, xi) = (Omega / (Omega + |xi|), xi) with a
// wrap-around halo of hx, hy points on each side, so that p +- l/2 needs no
// wrapping (FP32 arithmetic: the table is FP32, and GB300's FP64 division
// would dominate this kernel).  |xi| is floored at 1e-30 (sign kept).
// BF16X3 layout: float4 (alpha_q, alpha_q+1, xi_q, xi_q+1) for even q in the
// first half, for odd q in the second (the last entry repeated past the
// end): one thread per pair of entries 2t, 2t + 1 (one 8-byte load), which
// writes slot t of both halves, entry 2t + 2 from the next lane by a
// shuffle; 3xTF32: float2 (alpha_q, xi_q), one thread per entry.  Block 0
// also resets the work-item counter of the contraction that follows.
template <int PREC>
__global__ void __launch_bounds__(kTableBlock)
    scale_table_ext_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix,
                           int n, int* __restrict__ counter) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
  const int p = point_of(prefix, n, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const float omf = (float)pd.lam[0];
  const int n_ext = pd.n_ext;
  const int q = (blockIdx.x - prefix[p]) * kTableBlock + threadIdx.x;
  auto value = [&](float xi) {
    const float x = fmaxf(fabsf(xi), 1e-30f);
    return make_float2(__fdiv_rn(omf, omf + x), copysignf(x, xi));
  };
  auto entry = [&](int e) { return value(__ldg(pd.xiext + min(e, n_ext - 1))); };
  if constexpr (PREC == TUFRG_BF16X3) {
    const int half = (n_ext + 1) / 2;
    const int t = q;  // slot t of both halves: entries 2t, 2t + 1, 2t + 2
    // entries 2t, 2t + 1 (one 8-byte load where both exist; past the end the
    // last entry, as entry() clamps)
    float2 xi2;
    if (2 * t + 1 < n_ext) {
      xi2 = __ldg(reinterpret_cast<const float2*>(pd.xiext) + t);
    } else {
      const float v = __ldg(pd.xiext + min(2 * t, n_ext - 1));
      xi2 = make_float2(v, v);
    }
    const float2 e0 = value(xi2.x), e1 = value(xi2.y);
    // the CTA's threads cover consecutive t, every warp a run of 32
    float2 e2;
    e2.x = __shfl_down_sync(0xffffffffu, e0.x, 1);
    e2.y = __shfl_down_sync(0xffffffffu, e0.y, 1);
    if ((threadIdx.x & 31) == 31) e2 = entry(2 * t + 2);
    if (t < half) {
      pd.ext[t] = make_float4(e0.x, e1.x, e0.y, e1.y);
      pd.ext[half + t] = make_float4(e1.x, e2.x, e1.y, e2.y);
    }
  } else {
    if (q < n_ext) reinterpret_cast<float2*>(pd.ext)[q] = entry(q);
  }
}

}  // namespace

size_t tc_smem_bytes(int npad) {
  return 1024 + 2 * (4 * (size_t)kWTile + 2 * (size_t)npad * kRowBytes) + 128 + 8 * kRows;
}

int tc_k_per_block(int prec) { return prec == TUFRG_BF16X3 ? kRowBytes / 2 : kRowBytes / 4; }

int table_ctas(int n_ext, int prec) {
  const int threads = prec == TUFRG_BF16X3 ? (n_ext + 1) / 2 : n_ext;
  return (threads + kTableBlock - 1) / kTableBlock;
}

// Tensor maps of the two parts of F ([npad rows][kpad] elements, k
// contiguous): boxes of one K-block (128 bytes) by all npad rows, written
// with the 128-byte swizzle of the MMA's K-major operand layout.  The two
// 128-byte maps are stored one after the other in device memory.
tufrg_status make_f_tensor_maps(tufrg_ctx* c, cudaStream_t st) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return TUFRG_ERR_CUDA;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int es = c->p.precision == TUFRG_BF16X3 ? 2 : 4;
  CUtensorMap maps[2];
  const cuuint64_t dims[2] = {(cuuint64_t)c->tc_kpad, (cuuint64_t)c->tc_npad};
  const cuuint64_t strides[1] = {(cuuint64_t)c->tc_kpad * es};
  const cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / es), (cuuint32_t)c->tc_npad};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt =
      es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
  unsigned char* parts[2] = {c->d_Fhi, c->d_Flo};
  for (int t = 0; t < 2; ++t)
    if (encode(&maps[t], dt, 2, parts[t], dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return TUFRG_ERR_ARG;
  static_assert(sizeof(CUtensorMap) == 128, "two maps of 128 bytes");
  if (cudaMalloc(&c->d_tmap, sizeof(maps)) != cudaSuccess) return TUFRG_ERR_OOM;
  TUFRG_CUDA(cudaMemcpyAsync(c->d_tmap, maps, sizeof(maps), cudaMemcpyHostToDevice, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

tufrg_status prepare_loops_tc_multi(const MultiView& v) {
  const int smem = smem_optin();
  if ((int)tc_smem_bytes(v.npad_max) > smem) return TUFRG_ERR_ARG;
  if (v.tc_prec == TUFRG_BF16X3)
    TUFRG_CUDA(cudaFuncSetAttribute(loops_tc_kernel<TUFRG_BF16X3>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  else if (v.tc_prec == TUFRG_3XTF32)
    TUFRG_CUDA(cudaFuncSetAttribute(loops_tc_kernel<TUFRG_3XTF32>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return TUFRG_OK;
}

tufrg_status launch_loops_tc_multi(const MultiView& v, double* chi, cudaStream_t st) {
  TUFRG_CHECK(launch_loops_tc_rows_multi(v, st));
  return launch_expand_multi(v, chi, st);
}

tufrg_status launch_loops_tc_rows_multi(const MultiView& v, cudaStream_t st, cudaEvent_t* ev) {
  if (v.tc_prec == TUFRG_FP64 || v.n_items == 0) return TUFRG_ERR_ARG;
  if (v.tc_prec == TUFRG_BF16X3)
    scale_table_ext_kernel<TUFRG_BF16X3><<<v.total(kKindTable), kTableBlock, 0, st>>>(
        v.d, v.dprefix(kKindTable), v.n, v.d_counter);
  else
    scale_table_ext_kernel<TUFRG_3XTF32><<<v.total(kKindTable), kTableBlock, 0, st>>>(
        v.d, v.dprefix(kKindTable), v.n, v.d_counter);
  TUFRG_CUDA(cudaGetLastError());
  TcArgs a;
  a.pts = v.d;
  a.items = v.d_items;
  a.n_items = v.n_items;
  a.counter = v.d_counter;
  a.partial = v.d_partial;
  a.err = v.d_err;
  a.kbps = v.kbps;
  a.npad_max = v.npad_max;
  a.tmem_cols = v.tmem_cols;
  const int ctas = std::min(v.ctas, v.n_items);
  const size_t smem = tc_smem_bytes(v.npad_max);
  if (ev) TUFRG_CUDA(cudaEventRecord(ev[0], st));
  if (v.tc_prec == TUFRG_BF16X3)
    loops_tc_kernel<TUFRG_BF16X3><<<ctas, kThreads, smem, st>>>(a);
  else
    loops_tc_kernel<TUFRG_3XTF32><<<ctas, kThreads, smem, st>>>(a);
  TUFRG_CUDA(cudaGetLastError());
  if (ev) TUFRG_CUDA(cudaEventRecord(ev[1], st));
  return launch_tc_rows_multi(v, st);
}

}  // namespace tufrg
