// Step ii (Eq. chis) on the 5th-generation tensor cores (tcgen05, TMEM).
//
//   chi_dot_{pair}(l) = sum_k F_{pair}(k) W(k, l)
//
// as D[row = l-representative][n = pair] = sum_k W[row][k] F[n][k] with the
// operands split into high and low parts of a narrow type (BF16x3:
// bf16 hi/lo, kind::f16; 3xTF32: tf32 hi/lo, kind::tf32) and three products
// W_hi F_hi + W_lo F_hi + W_hi F_lo accumulated in FP32 in tensor memory;
// the split-K partial sums of each CTA are combined (fixed order, compensated
// FP32 pairs, FP64 result) by a second kernel.  The propagator operand W is
// generated in registers from the per-scale FP32 table (A = 1/(Omega + |xi|),
// u = xi A, extended by a wrap-around halo so p +- l/2 is one add from p)
// with the same closed-form frequency integral as the FP64 path, and written
// straight into the 128B-swizzled K-major shared-memory layout the MMA reads;
// F (scale independent) is staged with cp.async.  Both channels share W's
// table reads and divisions and have their own accumulator.
//
// Persistent CTAs (one per SM, 17 warps) take work items -- (point, tile of
// 128 l-rows, range of K-blocks) of any number of points -- from a queue
// ordered by cost.  Warps 0-15 produce the W tiles of a K-block (8 rows each,
// lanes along k, table loads of several rows in flight) and stage F, then
// read the accumulators out (warp w reads the 32 TMEM lanes 32 (w % 4).. of
// channel (w / 4) % 2, half of the columns).  Warp 16 owns TMEM and one of
// its threads issues the MMAs.  Two pipeline stages, mbarriers full/empty, whose phases
// run on across items; every wait is bounded in time and a timeout sets an
// error word, stops the pipeline, drains the issued MMAs and frees TMEM.
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
constexpr int kDepth = 4;           // producer units in flight (table gathers ahead)

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

template <int PREC>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
  if constexpr (PREC == TUFRG_BF16X3) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}


// Closed-form frequency integral of the two loops for two propagator pairs
// at once, with paired FP32 instructions, from the table values A and u of
// both propagators (a at p + l/2, b at p - l/2).  With x = |xi| = |u| / A and
// Omega A = 1 - |u|:
//   D = A_a A_b (5 Omega (A_a + A_b) - 3 - 2 Omega^2 (A_a^2 + A_a A_b + A_b^2))
//   S = (H_a + H_b) / (x_a + x_b),  H = x (3x + Omega) A^3 = |u| (1 + 2|u|) A,
//     = A_a A_b (H_a + H_b) / (|u_a| A_b + |u_b| A_a)
// the particle-particle weight is S for propagators of one sign, D else, and
// the particle-hole weight the other one.  The table holds |u| no smaller
// than 1e-30 (with the sign of xi): at x_a = x_b = 0 S is then A_a A_b =
// 1/Omega^2, its limit, and elsewhere the floor is far below FP32 resolution.
__device__ __forceinline__ void weights_au(const float2 Aa, const float2 usa, const float2 Ab,
                                           const float2 usb, float om, float om2, float2& wpp,
                                           float2& wph) {
  const float2 sa = __fadd2_rn(Aa, Ab), pa = __fmul2_rn(Aa, Ab);
  const float2 t1 = __ffma2_rn(sa, sa, make_float2(-pa.x, -pa.y));
  const float2 t2 = __ffma2_rn(make_float2(5.f * om, 5.f * om), sa, make_float2(-3.f, -3.f));
  const float2 br = __ffma2_rn(make_float2(-2.f * om2, -2.f * om2), t1, t2);
  const float2 D = __fmul2_rn(pa, br);
  const float2 ua = make_float2(fabsf(usa.x), fabsf(usa.y));
  const float2 ub = make_float2(fabsf(usb.x), fabsf(usb.y));
  const float2 ha = __fmul2_rn(ua, __ffma2_rn(ua, make_float2(2.f, 2.f), make_float2(1.f, 1.f)));
  const float2 hb = __fmul2_rn(ub, __ffma2_rn(ub, make_float2(2.f, 2.f), make_float2(1.f, 1.f)));
  const float2 num = __fmul2_rn(pa, __ffma2_rn(ha, Aa, __fmul2_rn(hb, Ab)));
  const float2 den = __ffma2_rn(ua, Ab, __fmul2_rn(ub, Aa));
  const float2 sg = __fmul2_rn(usa, usb);
  const float S0 = __fdividef(num.x, den.x), S1 = __fdividef(num.y, den.y);
  wpp = make_float2(sg.x > 0.f ? S0 : D.x, sg.y > 0.f ? S1 : D.y);
  wph = make_float2(sg.x > 0.f ? D.x : S0, sg.y > 0.f ? D.y : S1);
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
  int* counter;       // next item (zero before the launch)
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
  const uint32_t bar_full = ctrl, bar_empty = ctrl + 16, bar_done = ctrl + 32;
  unsigned char* gctrl = gbase + 2u * stage_bytes;
  volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(gctrl + 48);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(gctrl + 52);
  volatile int4* s_item = reinterpret_cast<volatile int4*>(gctrl + 64);
  int* s_off = reinterpret_cast<int*>(gctrl + 128);     // 3xTF32: row offsets
  int2* s_idx = reinterpret_cast<int2*>(gctrl + 128);   // BF16X3: row gather indices

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(bar_full + 8 * s, kProducers);
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
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = atomicAdd(a.counter, 1);
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
    const int row0 = tile * kRows;
    const int nvalid = min(kRows, pd.nrow - row0);  // rows of this tile with an l
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
    const double omd = pd.lam[0];
    const float om = (float)omd, om2 = (float)(omd * omd);

    if (warp < kProducers) {
      // ---------------------------------------------------------- producers
      // BF16X3: pairs (A_q, A_q+1, u_q, u_q+1) of even q at ext, of odd q at
      // ext + (n_ext + 1) / 2, read at the row's s_idx; 3xTF32: (A_q, u_q)
      // per point
      const float4* ext = pd.ext;
      const float2* ext2 = reinterpret_cast<const float2*>(pd.ext);
      const unsigned char* Fhi = pd.Fhi;
      const unsigned char* Flo = pd.Flo;
      const size_t frow = (size_t)pd.kpad_tc * P::kElem;  // bytes per F row
      const int fchunks = 8 * npad;  // 16-byte chunks per F tile
      // this warp's rows with an l, in units of kUnitRows rows
      const int nrw = max(0, min(kRows / kProducers, (nvalid - warp + kProducers - 1) / kProducers));
      const int nunits = (nrw + kUnitRows - 1) / kUnitRows;
      // The table gathers run kDepth - 1 units ahead of the arithmetic, in a
      // ring of register buffers, across K-block boundaries too (the gathers
      // of the next K-block's first units are issued while the last units of
      // this one are computed).  Every warp gathers all kUnits units of a
      // K-block (rows without an l read offset 0) and computes only those
      // with an l (the accumulator rows of the others are never read).
      using Buf = typename P::Buf;
      auto load_unit = [&](int u, int pb, Buf& b) {
        if constexpr (P::kPerLane == 2) {  // one row, two loop points: one pair each side
          const int2 ix = s_idx[warp + kProducers * u];
          const int hb = pb >> 1;
          b.v[0] = __ldg(ext + (hb + ix.x));
          b.v[1] = __ldg(ext + (hb + ix.y));
        } else {  // two rows, one loop point
          const int off0 = s_off[warp + kProducers * (2 * u)];
          const int off1 = s_off[warp + kProducers * (2 * u + 1)];
          b.v[0] = __ldg(ext2 + (pb + off0));
          b.v[1] = __ldg(ext2 + (pb - off0));
          b.v[2] = __ldg(ext2 + (pb + off1));
          b.v[3] = __ldg(ext2 + (pb - off1));
        }
      };
      auto do_unit = [&](int u, uint32_t st, const Buf& b) {
        float2 wpp, wph;
        if constexpr (P::kPerLane == 2)
          weights_au(make_float2(b.v[0].x, b.v[0].y), make_float2(b.v[0].z, b.v[0].w),
                     make_float2(b.v[1].x, b.v[1].y), make_float2(b.v[1].z, b.v[1].w), om, om2,
                     wpp, wph);
        else
          weights_au(make_float2(b.v[0].x, b.v[2].x), make_float2(b.v[0].y, b.v[2].y),
                     make_float2(b.v[1].x, b.v[3].x), make_float2(b.v[1].y, b.v[3].y), om, om2,
                     wpp, wph);
        if constexpr (PREC == TUFRG_BF16X3) {
          uint32_t v[4];
          const __nv_bfloat162 ph = __float22bfloat162_rn(wpp);
          const __nv_bfloat162 pl = __float22bfloat162_rn(
              __fadd2_rn(wpp, make_float2(-__low2float(ph), -__high2float(ph))));
          const __nv_bfloat162 hh = __float22bfloat162_rn(wph);
          const __nv_bfloat162 hl = __float22bfloat162_rn(
              __fadd2_rn(wph, make_float2(-__low2float(hh), -__high2float(hh))));
          std::memcpy(&v[0], &ph, 4);
          std::memcpy(&v[1], &pl, 4);
          std::memcpy(&v[2], &hh, 4);
          std::memcpy(&v[3], &hl, 4);
          // plain stores (the compiler may interleave the units around them);
          // the proxy fence before the stage's arrive orders them for the MMA
          unsigned char* dst = gbase + (st - base) + (warp + kProducers * u) * kRowBytes + swz;
#pragma unroll
          for (int t = 0; t < 4; ++t) *reinterpret_cast<uint32_t*>(dst + t * kWTile) = v[t];
        } else {
          const float w[2][2] = {{wpp.x, wph.x}, {wpp.y, wph.y}};
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            uint32_t v[4];
            v[0] = tf32_rna(w[j][0]);
            v[1] = tf32_rna(w[j][0] - __uint_as_float(v[0]));
            v[2] = tf32_rna(w[j][1]);
            v[3] = tf32_rna(w[j][1] - __uint_as_float(v[2]));
            unsigned char* dst =
                gbase + (st - base) + (warp + kProducers * (2 * u + j)) * kRowBytes + swz;
#pragma unroll
            for (int t = 0; t < 4; ++t) *reinterpret_cast<uint32_t*>(dst + t * kWTile) = v[t];
          }
        }
      };
      static_assert(kUnits % kDepth == 0, "the ring continues across K-blocks");
      Buf buf[kDepth];
      // this lane's first loop point of a K-block as an offset into the halo
      // table (padding points use a valid entry: their F is zero); BF16X3
      // lanes take loop points 2 lane, 2 lane + 1 of the K-block, neighbours
      // iy, iy + 1 of one column, i.e. table entries pb, pb + 1
      int pb = cnt > 0 ? __ldg(pd.kbase + kb0 * KB + P::kPerLane * lane) : 0;
#pragma unroll
      for (int t = 0; t < kDepth - 1; ++t)
        if (cnt > 0) load_unit(t, pb, buf[t]);
      for (int kb = 0; kb < cnt; ++kb) {
        const uint32_t gk = g + kb;
        const uint32_t s = gk & 1;
        if (gk >= 2 && !mbar_wait(bar_empty + 8 * s, ((gk >> 1) + 1) & 1)) {
          atomicOr(a.err, 1);
          *abort_flag = 1;
        }
        if (*abort_flag) break;
        const uint32_t st = base + s * stage_bytes;
        const int k0 = (kb0 + kb) * KB;
        const size_t fk = (size_t)k0 * P::kElem;
        for (int c = threadIdx.x; c < 2 * fchunks; c += 32 * kProducers) {
          const int t = c >= fchunks, rem = c - t * fchunks, row = rem >> 3, ch = rem & 7;
          cp_async16(st + 4u * kWTile + t * fmax + row * kRowBytes + ((ch ^ (row & 7)) << 4),
                     (t ? Flo : Fhi) + (size_t)row * frow + fk + ch * 16);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        // (after the item's last K-block the ring gathers this one's first
        // units again: valid addresses, no branch)
        const int pbn = kb + 1 < cnt ? __ldg(pd.kbase + k0 + KB + P::kPerLane * lane) : pb;
        // warps with all kUnits units run the K-block without a branch, so
        // the compiler can interleave the units' arithmetic
        auto kblock = [&](auto full) {
#pragma unroll
          for (int u = 0; u < kUnits; ++u) {
            const int t = u + kDepth - 1;  // unit gathered now, into the slot unit u - 1 freed
            if (t < kUnits)
              load_unit(t, pb, buf[t % kDepth]);
            else
              load_unit(t - kUnits, pbn, buf[t % kDepth]);
            if (decltype(full)::value || u < nunits) do_unit(u, st, buf[u % kDepth]);
          }
        };
        if (nunits == kUnits)
          kblock(std::true_type{});
        else
          kblock(std::false_type{});
        pb = pbn;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_full + 8 * s);
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
        if (!mbar_wait(bar_full + 8 * s, (gk >> 1) & 1)) {
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
            mma<PREC>(d, ah, bh, idesc, !(first && kk == 0));
            mma<PREC>(d, al, bh, idesc, 1);
            mma<PREC>(d, ah, bl, idesc, 1);
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
      const bool ok = mbar_wait(bar_done, j & 1);
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
#pragma unroll
          for (int e = 0; e < 16; ++e) out[(size_t)(c0 + e) * pd.nrow_pad] = acc[e];
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

// Per-scale FP32 table (A, u) = (1/(Omega + |xi|), xi A) with a wrap-around
// halo of hx, hy points on each side, so that p +- l/2 needs no wrapping
// (FP32 arithmetic: the table is FP32, and GB300's FP64 division would
// dominate this kernel).  |u| is floored at 1e-30 (sign of xi kept).  BF16X3
// layout: float4 (A_q, A_q+1, u_q, u_q+1) for even q in the first half, for
// odd q in the second (the last entry repeated past the end); 3xTF32: float2
// (A_q, u_q).  One thread per entry q, the neighbour's values by a shuffle.
// Block 0 also resets the work-item counter of the contraction that follows.
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
  auto entry = [&](int e) {
    const float xi = __ldg(pd.xiext + min(e, n_ext - 1));
    const float A = __frcp_rn(omf + fabsf(xi));
    return make_float2(A, copysignf(fmaxf(fabsf(xi * A), 1e-30f), xi));
  };
  const float2 a = entry(q);
  if constexpr (PREC == TUFRG_BF16X3) {
    const int half = (n_ext + 1) / 2;
    // the CTA's threads cover consecutive q, every warp a run of 32
    float2 b;
    b.x = __shfl_down_sync(0xffffffffu, a.x, 1);
    b.y = __shfl_down_sync(0xffffffffu, a.y, 1);
    if ((threadIdx.x & 31) == 31) b = entry(q + 1);
    if (q < 2 * half) pd.ext[(q & 1) * half + (q >> 1)] = make_float4(a.x, b.x, a.y, b.y);
  } else {
    if (q < n_ext) reinterpret_cast<float2*>(pd.ext)[q] = a;
  }
}

}  // namespace

size_t tc_smem_bytes(int npad) {
  return 1024 + 2 * (4 * (size_t)kWTile + 2 * (size_t)npad * kRowBytes) + 128 + 8 * kRows;
}

int tc_k_per_block(int prec) { return prec == TUFRG_BF16X3 ? kRowBytes / 2 : kRowBytes / 4; }

int table_ctas(int n_ext) { return (n_ext + 1 + kTableBlock - 1) / kTableBlock; }

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
