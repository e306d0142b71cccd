// Host-side construction of the scale-independent device tables.
//
// * dispersion table xi(p) on the fine grid (Eq. hubb-disp);
// * loop points: half of the fine grid, one point of each pair (p, -p) with
//   weight 2 (weight 1 for p = -p).  The loop integrand f_m f_n w is even
//   under p -> -p for parity-allowed pairs (pi_m pi_n = +1) and the others
//   vanish (App. C), so the sum runs over half the zone;
// * F[pair][k] = weight_k f_m(p_k) f_n(p_k) / Nf for the allowed pairs m <= n;
// * loop rows: one per class of l under the point-group elements that map l
//   into the zone without a fold (C4v orbits of interior l, classes of up to
//   four zone-boundary l; {l, -l} off square grids) with the half-shift of
//   the row's l on the fine grid (l/2 lands on the fine grid when
//   nf % (2 nc) == 0 and nf % 4 == 0) and the list of (l, g) it serves;
// * position-space projection data (Sec. 2.5: the Kronecker-delta overlaps
//   and Fourier phases are scale independent and computed once).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "internal.h"

namespace tufrg {
namespace {

constexpr int kKC = 16;            // loop points per chunk of the FP64 loop kernel
constexpr int kLT = 32;            // l per CTA of the FP64 loop kernel
constexpr int kTargetCTAs = 4 * 152;

// bf16 of a float by round to nearest even (finite inputs)
uint16_t bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// tf32 of a float: 10 explicit mantissa bits, rounded half away from zero
uint32_t tf32_rna(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (u + 0x1000u) & 0xFFFFE000u;
}

int imod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Cross-projection signatures.  For target channel T with projection rule
// (k1, k2, k3)(l, k, k') of Eqs. (proj-P/C/D) and source channel S whose
// folded bosonic momentum is l' = fold(k +- k'), put k' = s (l' - k).  The
// fermionic arguments of Phi^S then read q = k + l/2 - l'/2 and
// q' = sq k + bq l/2 + gq l'/2.  With f(k) = sum_R c(R) e^{ik.R} the k sum
// forces R1 - s R2 + R3 + sq R4 = 0 (mod the coarse grid), the source enters
// through its Fourier series at X = s R2 + (-R3 + gq R4)/2 and the result
// carries the phase e^{i l.Y}, Y = (R3 + bq R4)/2.
struct Sig {
  int target, source, s, sq, bq, gq;
};
const Sig kSigs[6] = {
    {0, 1, +1, -1, +1, +1},  // P <- C : q' = -k + l/2 + l'/2
    {0, 2, -1, -1, +1, +1},  // P <- D
    {1, 0, +1, -1, +1, +1},  // C <- P
    {1, 2, -1, +1, -1, -1},  // C <- D : q' = k - l/2 - l'/2
    {2, 0, +1, +1, -1, -1},  // D <- P
    {2, 1, -1, +1, -1, -1},  // D <- C
};

template <class T>
tufrg_status upload(T** dptr, const std::vector<T>& h, cudaStream_t st) {
  size_t bytes = std::max<size_t>(h.size(), 1) * sizeof(T);
  if (cudaMalloc((void**)dptr, bytes) != cudaSuccess) return TUFRG_ERR_OOM;
  if (!h.empty()) TUFRG_CUDA(cudaMemcpyAsync(*dptr, h.data(), h.size() * sizeof(T),
                                             cudaMemcpyHostToDevice, st));
  return TUFRG_OK;
}

template <class T>
tufrg_status alloc(T** dptr, size_t n) {
  if (cudaMalloc((void**)dptr, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess)
    return TUFRG_ERR_OOM;
  return TUFRG_OK;
}

void build_proj(tufrg_ctx* c) {
  const Basis& B = c->basis;
  const int nb = B.nb;
  ProjTables& P = c->proj;
  std::map<std::array<int, 5>, int> keys;
  std::vector<std::vector<std::array<int, 4>>> rows[3];
  for (int t = 0; t < 3; ++t) rows[t].assign((size_t)nb * nb, {});
  int dmax = 0;
  for (const Sig& g : kSigs) {
    for (int b1 = 0; b1 < nb; ++b1)
      for (int b2 = 0; b2 < nb; ++b2)
        for (int b3 = 0; b3 < nb; ++b3)
          for (int b4 = 0; b4 < nb; ++b4) {
            int kx = B.bx[b1] - g.s * B.bx[b2] + B.bx[b3] + g.sq * B.bx[b4];
            int ky = B.by[b1] - g.s * B.by[b2] + B.by[b3] + g.sq * B.by[b4];
            if (imod(kx, c->ncx) != 0 || imod(ky, c->ncy) != 0) continue;
            int x2x = 2 * g.s * B.bx[b2] - B.bx[b3] + g.gq * B.bx[b4];
            int x2y = 2 * g.s * B.by[b2] - B.by[b3] + g.gq * B.by[b4];
            int y2x = B.bx[b3] + g.bq * B.bx[b4];
            int y2y = B.by[b3] + g.bq * B.by[b4];
            dmax = std::max({dmax, std::abs(x2x), std::abs(x2y), std::abs(y2x), std::abs(y2y)});
            auto ins = keys.emplace(std::array<int, 5>{g.source, b3, b4, x2x, x2y},
                                    (int)keys.size());
            // V = V0 - Phi^SC + Phi^C + Phi^D (Eq. simple-deco)
            rows[g.target][(size_t)b1 * nb + b2].push_back(
                {ins.first->second, y2x, y2y, g.source == 0 ? -1 : 1});
          }
  }
  P.dmax = dmax;
  P.nkeys = (int)keys.size();
  P.key_src.assign(P.nkeys, 0);
  P.key_b3.assign(P.nkeys, 0);
  P.key_b4.assign(P.nkeys, 0);
  P.key_dx.assign(P.nkeys, 0);
  P.key_dy.assign(P.nkeys, 0);
  for (auto& kv : keys) {
    int i = kv.second;
    P.key_src[i] = kv.first[0];
    P.key_b3[i] = kv.first[1];
    P.key_b4[i] = kv.first[2];
    P.key_dx[i] = kv.first[3];
    P.key_dy[i] = kv.first[4];
  }
  for (int t = 0; t < 3; ++t) {
    P.row_ptr[t].assign((size_t)nb * nb + 1, 0);
    P.term_key[t].clear();
    P.term_dx[t].clear();
    P.term_dy[t].clear();
    P.term_sign[t].clear();
    for (size_t o = 0; o < rows[t].size(); ++o) {
      for (auto& e : rows[t][o]) {
        P.term_key[t].push_back(e[0]);
        P.term_dx[t].push_back(e[1]);
        P.term_dy[t].push_back(e[2]);
        P.term_sign[t].push_back((double)e[3]);
      }
      P.row_ptr[t][o + 1] = (int)P.term_key[t].size();
    }
  }
  // the terms of each target grouped by phase position Y (in the order of
  // (2Y_x, 2Y_y)), within a position by output pair, within a pair in the
  // order above; padded to the same number of slots per position
  std::vector<std::vector<int4>> groups;
  P.gy.clear();
  for (int t = 0; t < 3; ++t) {
    P.gy_off[t] = (int)P.gy.size();
    std::map<std::pair<int, int>, std::vector<int4>> by_y;  // (o, key, sign, 0)
    for (int o = 0; o < nb * nb; ++o)
      for (int k = P.row_ptr[t][o]; k < P.row_ptr[t][o + 1]; ++k)
        by_y[{P.term_dx[t][k], P.term_dy[t][k]}].push_back(
            make_int4(o, P.term_key[t][k], P.term_sign[t][k] < 0 ? -1 : 1, 0));
    for (auto& kv : by_y) {
      P.gy.push_back(make_int2(kv.first.first, kv.first.second));
      groups.push_back(kv.second);
    }
  }
  P.gy_off[3] = (int)P.gy.size();
  P.gmaxt = 1;
  for (const auto& g : groups) P.gmaxt = std::max(P.gmaxt, (int)g.size());
  P.gslot.assign(groups.size() * P.gmaxt, make_int4(-1, -1, 0, 0));
  for (size_t g = 0; g < groups.size(); ++g)
    for (size_t k = 0; k < groups[g].size(); ++k) P.gslot[g * P.gmaxt + k] = groups[g][k];
}

}  // namespace

tufrg_status setup_proj(tufrg_ctx* c, cudaStream_t st);

tufrg_status setup_device(tufrg_ctx* c, cudaStream_t st, const SetupShare& share) {
  const Basis& B = c->basis;
  const int nff = c->nff, nb = c->nb;
  const double two_pi = 2.0 * M_PI;

  // dispersion on the fine grid, index ix * nfy + iy, p = -pi + 2 pi i / nf
  std::vector<double> cx(c->nfx), cy(c->nfy);
  for (int i = 0; i < c->nfx; ++i) cx[i] = std::cos(-M_PI + two_pi * i / c->nfx);
  for (int i = 0; i < c->nfy; ++i) cy[i] = std::cos(-M_PI + two_pi * i / c->nfy);
  std::vector<double4_32a> tab((size_t)c->nf);
  for (int ix = 0; ix < c->nfx; ++ix)
    for (int iy = 0; iy < c->nfy; ++iy) {
      double xi = -2.0 * c->p.t * (cx[ix] + cy[iy]) - 4.0 * c->p.tp * cx[ix] * cy[iy] - c->p.mu;
      tab[(size_t)ix * c->nfy + iy] = make_double4_32a(xi, 0.0, 0.0, 0.0);
    }
  TUFRG_CHECK(upload(&c->d_tab, tab, st));

  // loop points over half the zone, one of each pair {p, -p}: the columns
  // 0 < ix < nfx/2 whole, and the two self-partnered columns ix = 0, nfx/2
  // for 0 <= iy <= nfy/2.  Every run of consecutive loop points is a run of
  // consecutive iy, i.e. of consecutive entries of the [ix][iy] tables.
  std::vector<int2> kp;
  std::vector<double> kw;
  const int hy = c->nfy / 2, hx = c->nfx / 2;
  for (int ix = 1; ix < hx; ++ix)
    for (int iy = 0; iy < c->nfy; ++iy) {
      kp.push_back(make_int2(ix, iy));
      kw.push_back(2.0);
    }
  for (int ix : {0, hx}) {
    for (int iy = 0; iy <= hy; ++iy) {
      kp.push_back(make_int2(ix, iy));
      kw.push_back((iy == 0 || iy == hy) ? 1.0 : 2.0);
    }
    // columns of even length, so that loop points 2j, 2j + 1 are always
    // neighbours iy, iy + 1 of one column (the BF16X3 producers read them as
    // a pair): a padding point of weight 0
    if ((hy + 1) % 2) {
      kp.push_back(make_int2(ix, hy + 1));
      kw.push_back(0.0);
    }
  }
  c->kdim = (int)kp.size();

  // parity-allowed pairs m <= n
  c->pair_m.clear();
  c->pair_n.clear();
  for (int m = 0; m < nff; ++m)
    for (int n = m; n < nff; ++n)
      if (B.ff[m].parity * B.ff[n].parity == 1) {
        c->pair_m.push_back(m);
        c->pair_n.push_back(n);
      }
  c->npair = (int)c->pair_m.size();

  // Rows of the loop contraction and the l each row serves.  The loops are
  // covariant, chi(g l) = R^g chi(l) R^g^T with f(g k) = R^g f(k) (App. C;
  // xi is C4v symmetric), for every point-group element g that maps l into
  // the zone [-pi, pi)^2 without a fold: the folded g l then has the half
  // momentum g l/2.  For l inside the zone that is every g.  For l on the
  // zone boundary (a component at -pi) it is the elements that keep each -pi
  // component at -pi (four of eight for one such component, two for l =
  // (-pi, -pi)); the others send it to +pi, whose fold moves the half
  // momentum by pi.  These relations are closed under inverse and product,
  // so one row serves each class.  On square grids with a basis whose R^g
  // are signed permutations g ranges over C4v; otherwise over {e, -1}
  // (R^g = diag(parity), which leaves the parity-allowed loops unchanged).
  std::vector<int> symperm, symsign;
  const bool c4v = c->ncx == c->ncy && c->nfx == c->nfy && B.point_group(symperm, symsign);
  if (!c4v) {
    symperm.assign(8 * (size_t)nff, 0);
    symsign.assign(8 * (size_t)nff, 1);
    for (int g = 0; g < 8; ++g)
      for (int m = 0; m < nff; ++m) symperm[(size_t)g * nff + m] = m;
  }
  std::vector<int2> rowshift, rowimg;
  std::vector<int> rowimg_ptr(1, 0);
  std::vector<char> served(c->nl, 0);
  const int hcx = c->ncx / 2, hcy = c->ncy / 2;
  // A non-uniform mesh: the same classes on the mesh's lattice (u = j - nc m
  // / 2), where g serves l when the image g l is a mesh point with the same
  // two quadrature weights (then the projections of a covariant state are
  // covariant too); l/2 in fine-grid steps (-pi/2 + pi j / (nc m)) / (2 pi / nf)
  if (c->mesh) {
    const int div = c->ncx * c->mesh_m, hd = div / 2;
    std::map<std::pair<int, int>, int> at;
    for (int l = 0; l < c->nl; ++l) at[{c->mesh_pts[l].x, c->mesh_pts[l].y}] = l;
    const double* wp = c->mesh_w.data();
    const double* wc = wp + c->nl;
    for (int l = 0; l < c->nl; ++l) {
      if (served[l]) continue;
      const int ux = c->mesh_pts[l].x - hd, uy = c->mesh_pts[l].y - hd;
      for (int g = 0; g < 8; ++g) {
        if (!c4v && g != 0 && g != 2) continue;
        const int vx = kC4v[g][0][0] * ux + kC4v[g][0][1] * uy;
        const int vy = kC4v[g][1][0] * ux + kC4v[g][1][1] * uy;
        if (vx < -hd || vx >= div - hd || vy < -hd || vy >= div - hd) continue;
        const auto it = at.find({vx + hd, vy + hd});
        if (it == at.end()) continue;
        const int lg = it->second;
        if (served[lg] || wp[lg] != wp[l] || wc[lg] != wc[l]) continue;
        served[lg] = 1;
        rowimg.push_back(make_int2(lg, c4v ? g : 0));
      }
      rowimg_ptr.push_back((int)rowimg.size());
      rowshift.push_back(make_int2(-c->nfx / 4 + c->mesh_pts[l].x * (c->nfx / (2 * div)),
                                   -c->nfy / 4 + c->mesh_pts[l].y * (c->nfy / (2 * div))));
    }
  }
  for (int jx = 0; !c->mesh && jx < c->ncx; ++jx)
    for (int jy = 0; jy < c->ncy; ++jy) {
      const int l = jx * c->ncy + jy;
      if (served[l]) continue;
      for (int g = 0; g < 8; ++g) {
        if (!c4v && g != 0 && g != 2) continue;
        // g acts on u = j - n/2 (k = 2 pi u / n, u in [-n/2, n/2)); an image
        // outside that range would need a fold
        const int ux = jx - hcx, uy = jy - hcy;
        const int vx = kC4v[g][0][0] * ux + kC4v[g][0][1] * uy;
        const int vy = kC4v[g][1][0] * ux + kC4v[g][1][1] * uy;
        if (vx < -hcx || vx >= c->ncx - hcx || vy < -hcy || vy >= c->ncy - hcy) continue;
        const int lg = (vx + hcx) * c->ncy + (vy + hcy);
        if (served[lg]) continue;
        served[lg] = 1;
        rowimg.push_back(make_int2(lg, c4v ? g : 0));
      }
      rowimg_ptr.push_back((int)rowimg.size());
      // l/2 in fine-grid steps: (-pi/2 + pi j / nc) / (2 pi / nf)
      rowshift.push_back(make_int2(-c->nfx / 4 + jx * (c->nfx / (2 * c->ncx)),
                                   -c->nfy / 4 + jy * (c->nfy / (2 * c->ncy))));
    }
  c->nrow = (int)rowshift.size();
  c->shard_lo = 0;
  c->shard_hi = c->nrow;
  c->c4v = c4v;
  std::vector<int2> lrow(c->nl);
  for (int r = 0; r < c->nrow; ++r)
    for (int i = rowimg_ptr[r]; i < rowimg_ptr[r + 1]; ++i)
      lrow[rowimg[i].x] = make_int2(r, rowimg[i].y);

  c->rm = c->npair <= 16 ? 1 : (c->npair <= 32 ? 2 : 4);
  const int mt = 16 * c->rm;
  c->mtiles = (c->npair + mt - 1) / mt;
  c->mpad = c->mtiles * mt;
  const int ltiles = (c->nrow + kLT - 1) / kLT;
  const int nchunks = (c->kdim + kKC - 1) / kKC;
  // at most one wave of resident CTAs (4 per SM at 128 registers per thread)
  int ksplit = std::max(1, kTargetCTAs / (ltiles * c->mtiles));
  ksplit = std::min(ksplit, nchunks);
  c->kchunk = ((nchunks + ksplit - 1) / ksplit) * kKC;
  c->ksplit = (c->kdim + c->kchunk - 1) / c->kchunk;
  c->kpad = c->ksplit * c->kchunk;

  const tufrg_ctx* dl = share.loops;
  c->borrowed_loops = dl != nullptr;
  if (dl) {  // same grids, bonds and precision: the scale-independent loop tables
    c->d_kidx = dl->d_kidx;
    c->d_F = dl->d_F;
    c->d_pair = dl->d_pair;
    c->d_pairidx = dl->d_pairidx;
    c->d_rowoff = dl->d_rowoff;
    c->d_kbase = dl->d_kbase;
    c->d_Fhi = dl->d_Fhi;
    c->d_Flo = dl->d_Flo;
    c->d_tmap = dl->d_tmap;
    c->d_shift = dl->d_shift;
    c->d_rowimg_ptr = dl->d_rowimg_ptr;
    c->d_rowimg = dl->d_rowimg;
    c->d_lrow = dl->d_lrow;
    c->d_lgather = dl->d_lgather;
    c->d_symperm = dl->d_symperm;
    c->d_symsign = dl->d_symsign;
  }
  std::vector<int2> kidx(c->kpad, make_int2(-1, -1));
  for (int k = 0; k < c->kdim; ++k) kidx[k] = kp[k];
  if (!dl) TUFRG_CHECK(upload(&c->d_kidx, kidx, st));

  // form factors at the loop points via per-direction cos/sin tables
  const int R = 4;
  std::vector<double> fv(dl ? 0 : (size_t)nff * c->kdim);
  for (int k = 0; k < (dl ? 0 : c->kdim); ++k) {
    double px = -M_PI + two_pi * kp[k].x / c->nfx, py = -M_PI + two_pi * kp[k].y / c->nfy;
    double cxr[R], sxr[R], cyr[R], syr[R];
    for (int r = 0; r < R; ++r) {
      cxr[r] = std::cos(r * px);
      sxr[r] = std::sin(r * px);
      cyr[r] = std::cos(r * py);
      syr[r] = std::sin(r * py);
    }
    for (int m = 0; m < nff; ++m) {
      double v = 0.0;
      for (const TrigTerm& t : B.ff[m].terms) {
        int ax = std::abs(t.rx), ay = std::abs(t.ry);
        double ccx = cxr[ax], ssx = t.rx < 0 ? -sxr[ax] : sxr[ax];
        double ccy = cyr[ay], ssy = t.ry < 0 ? -syr[ay] : syr[ay];
        double val = t.is_sin ? (ssx * ccy + ccx * ssy) : (ccx * ccy - ssx * ssy);
        v += t.coef * val;
      }
      fv[(size_t)m * c->kdim + k] = v;
    }
  }
  std::vector<double> F(dl ? 0 : (size_t)c->mpad * c->kpad, 0.0);
  std::vector<int> pair(c->mpad, -1);
  for (int q = 0; q < c->npair; ++q) {
    int m = c->pair_m[q], n = c->pair_n[q];
    pair[q] = m * nff + n;
    for (int k = 0; k < (dl ? 0 : c->kdim); ++k)
      F[(size_t)q * c->kpad + k] =
          kw[k] * fv[(size_t)m * c->kdim + k] * fv[(size_t)n * c->kdim + k] / c->nf;
  }
  std::vector<int> pairidx((size_t)nff * nff, -1);
  for (int q = 0; q < c->npair; ++q) {
    pairidx[(size_t)c->pair_m[q] * nff + c->pair_n[q]] = q;
    pairidx[(size_t)c->pair_n[q] * nff + c->pair_m[q]] = q;
  }
  if (!dl) {
    TUFRG_CHECK(upload(&c->d_F, F, st));
    TUFRG_CHECK(upload(&c->d_pair, pair, st));
    TUFRG_CHECK(upload(&c->d_pairidx, pairidx, st));
  }

  if (c->p.precision != TUFRG_FP64) {
    // tensor-core path: M = 128 l-rows per tile, N = pairs (multiple of 16),
    // K-blocks of one 128-byte swizzle row (the split of the K-blocks into
    // work items belongs to the context's multi-point view)
    const int kb = tc_k_per_block(c->p.precision);
    c->tc_npad = (c->npair + 15) / 16 * 16;
    if (c->tc_npad > 176) return TUFRG_ERR_ARG;  // two pipeline stages must fit shared memory
    c->tc_nrow_pad = (c->nrow + 127) / 128 * 128;
    c->tc_nkb = (c->kdim + kb - 1) / kb;
    c->tc_kpad = c->tc_nkb * kb;
    // accumulator sets: as many (<= 4) as fit the 512 TMEM columns
    c->tc_nsets = 1;
    while (c->tc_nsets < 4 && 2 * c->tc_nsets * 2 * c->tc_npad <= 512) c->tc_nsets *= 2;
    // halo table (offsets of p + l/2 below)
    c->tc_hx = c->nfx / 4;
    c->tc_hy = c->nfy / 4;
    c->tc_wy = c->nfy + 2 * c->tc_hy;
    // (A, xi A) per point: BF16X3 as two float4 arrays of point pairs
    // (2j, 2j + 1) and (2j + 1, 2j + 2), 3xTF32 as one float2 per point
    const size_t n_ext = (size_t)(c->nfx + 2 * c->tc_hx) * c->tc_wy;
    TUFRG_CHECK(alloc(&c->d_ext, 2 * ((n_ext + 1) / 2)));
    // the scale-independent xi at every point of the halo table (wrapped)
    std::vector<float> xiext(n_ext);
    for (size_t e = 0; e < n_ext; ++e) {
      const int ix = imod((int)(e / c->tc_wy) - c->tc_hx, c->nfx);
      const int iy = imod((int)(e % c->tc_wy) - c->tc_hy, c->nfy);
      xiext[e] = (float)tab[(size_t)ix * c->nfy + iy].x;
    }
    TUFRG_CHECK(upload(&c->d_xiext, xiext, st));
  }
  if (c->p.precision != TUFRG_FP64 && !dl) {
    const bool bf16 = c->p.precision == TUFRG_BF16X3;
    const int es = bf16 ? 2 : 4;
    std::vector<int> rowoff(c->nrow);
    for (int r = 0; r < c->nrow; ++r) rowoff[r] = rowshift[r].x * c->tc_wy + rowshift[r].y;
    TUFRG_CHECK(upload(&c->d_rowoff, rowoff, st));
    std::vector<int> kbase(c->tc_kpad, c->tc_hx * c->tc_wy + c->tc_hy);  // padding: centre
    for (int k = 0; k < c->kdim; ++k)
      kbase[k] = (kp[k].x + c->tc_hx) * c->tc_wy + kp[k].y + c->tc_hy;
    TUFRG_CHECK(upload(&c->d_kbase, kbase, st));
    std::vector<unsigned char> fh((size_t)c->tc_npad * c->tc_kpad * es, 0);
    std::vector<unsigned char> fl(fh.size(), 0);
    for (int q = 0; q < c->npair; ++q)
      for (int k = 0; k < c->kdim; ++k) {
        const float f = (float)F[(size_t)q * c->kpad + k];
        const size_t off = ((size_t)q * c->tc_kpad + k) * es;
        if (bf16) {
          const uint16_t h = bf16_rne(f);
          const uint16_t l = bf16_rne(f - bf16_value(h));
          std::memcpy(&fh[off], &h, 2);
          std::memcpy(&fl[off], &l, 2);
        } else {
          const uint32_t h = tf32_rna(f);
          float hf;
          std::memcpy(&hf, &h, 4);
          const uint32_t l = tf32_rna(f - hf);
          std::memcpy(&fh[off], &h, 4);
          std::memcpy(&fl[off], &l, 4);
        }
      }
    TUFRG_CHECK(upload(&c->d_Fhi, fh, st));
    TUFRG_CHECK(upload(&c->d_Flo, fl, st));
    TUFRG_CHECK(make_f_tensor_maps(c, st));
  }
  TUFRG_CHECK(alloc(&c->d_err, 1));
  TUFRG_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));

  // analytic-xi mode: l/2 off the fine grid (nf not a multiple of 2 nc); the
  // FP64 loops take xi(p +- l/2) from per-row cosine tables (the row's
  // representative l = (jx, jy), l/2 = -pi/2 + pi j / nc)
  c->analytic = (c->nfx % (2 * c->ncx)) != 0 || (c->nfy % (2 * c->ncy)) != 0;
  if (dl) {
    c->d_acos = dl->d_acos;
  } else if (c->analytic) {
    const int alen = 2 * (c->nfx + c->nfy);
    std::vector<double> ac((size_t)c->nrow * alen);
    for (int r = 0; r < c->nrow; ++r) {
      const int l = rowimg[rowimg_ptr[r]].x, jx = l / c->ncy, jy = l % c->ncy;
      const double hx = -0.5 * M_PI + M_PI * jx / c->ncx, hy = -0.5 * M_PI + M_PI * jy / c->ncy;
      double* row = ac.data() + (size_t)r * alen;
      for (int i = 0; i < c->nfx; ++i) {
        const double px = -M_PI + two_pi * i / c->nfx;
        row[i] = std::cos(px + hx);
        row[c->nfx + i] = std::cos(px - hx);
      }
      for (int i = 0; i < c->nfy; ++i) {
        const double py = -M_PI + two_pi * i / c->nfy;
        row[2 * c->nfx + i] = std::cos(py + hy);
        row[2 * c->nfx + c->nfy + i] = std::cos(py - hy);
      }
    }
    TUFRG_CHECK(upload(&c->d_acos, ac, st));
  }
  if (!dl) {
    TUFRG_CHECK(upload(&c->d_shift, rowshift, st));
    TUFRG_CHECK(upload(&c->d_rowimg_ptr, rowimg_ptr, st));
    TUFRG_CHECK(upload(&c->d_rowimg, rowimg, st));
    TUFRG_CHECK(upload(&c->d_lrow, lrow, st));
    // entry (m, n) of the loops of l = s_m s_n chi(row)_{p(m) p(n)} for the
    // row serving l and its group element's signed permutation
    std::vector<int> lgather((size_t)c->nl * nff * nff, 0);
    for (int l = 0; l < c->nl; ++l) {
      const int r = lrow[l].x, g = lrow[l].y;
      for (int m = 0; m < nff; ++m)
        for (int n = 0; n < nff; ++n) {
          const int q = pairidx[(size_t)symperm[(size_t)g * nff + m] * nff +
                                symperm[(size_t)g * nff + n]];
          if (q < 0) continue;
          const int sg = symsign[(size_t)g * nff + m] * symsign[(size_t)g * nff + n];
          lgather[((size_t)l * nff + m) * nff + n] = sg * (r * c->npair + q + 1);
        }
    }
    TUFRG_CHECK(upload(&c->d_lgather, lgather, st));
    TUFRG_CHECK(upload(&c->d_symperm, symperm, st));
    TUFRG_CHECK(upload(&c->d_symsign, symsign, st));
  }

  const tufrg_ctx* dp = share.proj;
  c->borrowed_proj = dp != nullptr;
  if (dp) {  // same coarse grid and bonds: the projection tables
    c->proj = dp->proj;
    c->d_coef = dp->d_coef;
    c->d_phase = dp->d_phase;
    c->d_coef_f = dp->d_coef_f;
    c->d_phase_f = dp->d_phase_f;
    c->d_yphase = dp->d_yphase;
    c->d_yphase_f = dp->d_yphase_f;
    c->d_row_ptr = dp->d_row_ptr;
    c->d_terms = dp->d_terms;
    for (int t = 0; t < 3; ++t) c->term_off[t] = dp->term_off[t];
    c->n_terms = dp->n_terms;
    c->d_gslot = dp->d_gslot;
  } else {
    TUFRG_CHECK(setup_proj(c, st));
  }
  const ProjTables& P = c->proj;

  // workspace
  TUFRG_CHECK(alloc(&c->d_lambda, 4));
  if (share.workspace) {
    TUFRG_CHECK(alloc(&c->d_partial, (size_t)c->ksplit * 2 * c->mpad * c->nrow));
    TUFRG_CHECK(alloc(&c->d_chi, (size_t)2 * c->nl * nff * nff));
    TUFRG_CHECK(alloc(&c->d_V, (size_t)3 * c->nl * nff * nff));
    if (c->p.precision != TUFRG_FP64) TUFRG_CHECK(alloc(&c->d_y32, (size_t)3 * c->nl * nff * nff));
    TUFRG_CHECK(alloc(&c->d_bt, ctx_bt_elems(c)));
    TUFRG_CHECK(alloc(&c->d_fkey, fkey_elems(2 * P.dmax + 1, nb)));
    // the loop kernels write only the parity-allowed pairs
    TUFRG_CUDA(cudaMemsetAsync(c->d_chi, 0, sizeof(double) * 2 * c->nl * nff * nff, st));
    TUFRG_CUDA(cudaStreamCreateWithFlags(&c->fstream, cudaStreamNonBlocking));
    TUFRG_CUDA(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    TUFRG_CUDA(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    TUFRG_CUDA(cudaStreamCreateWithFlags(&c->pstream, cudaStreamNonBlocking));
    TUFRG_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    TUFRG_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    TUFRG_CUDA(cudaEventCreateWithFlags(&c->ev_stage, cudaEventDisableTiming));
  }
  if (share.own_view) {
    double* lam[1] = {c->d_lambda};
    tufrg_ctx* self[1] = {c};
    TUFRG_CHECK(view_build(c->view, self, 1, lam, nullptr, c->d_err, c->p.precision, 0, st));
  }
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

// bond coefficients and the position-space projection tables
tufrg_status setup_proj(tufrg_ctx* c, cudaStream_t st) {
  const Basis& B = c->basis;
  const int nff = c->nff, nb = c->nb;
  std::vector<double2> coef((size_t)nff * nb);
  for (size_t i = 0; i < coef.size(); ++i)
    coef[i] = make_double2(B.coef[i].real(), B.coef[i].imag());
  TUFRG_CHECK(upload(&c->d_coef, coef, st));
  std::vector<float2> coef_f(coef.size());
  for (size_t i = 0; i < coef.size(); ++i)
    coef_f[i] = make_float2((float)coef[i].x, (float)coef[i].y);
  TUFRG_CHECK(upload(&c->d_coef_f, coef_f, st));

  build_proj(c);
  const ProjTables& P = c->proj;
  const int nd = 2 * P.dmax + 1;
  std::vector<double2> phase((size_t)(c->ncx + c->ncy) * nd);
  for (int dim = 0; dim < 2; ++dim) {
    int n = dim == 0 ? c->ncx : c->ncy, off = dim == 0 ? 0 : c->ncx;
    for (int i = 0; i < n; ++i)
      for (int d = -P.dmax; d <= P.dmax; ++d) {
        // l = pi (2i - n)/n, position d/2:  l * d/2 = pi (2i - n) d / (2n)
        double a = M_PI * (double)((2 * i - n) * d) / (2.0 * n);
        phase[(size_t)(off + i) * nd + d + P.dmax] = make_double2(std::cos(a), std::sin(a));
      }
  }
  TUFRG_CHECK(upload(&c->d_phase, phase, st));
  std::vector<float2> phase_f(phase.size());
  for (size_t i = 0; i < phase.size(); ++i)
    phase_f[i] = make_float2((float)phase[i].x, (float)phase[i].y);
  TUFRG_CHECK(upload(&c->d_phase_f, phase_f, st));
  // keys numbered densely over (source, 2X_x, 2X_y, b3, b4): the Fourier
  // values of all keys at a position X come from one DFT of the state
  std::vector<int> dense(P.nkeys);
  for (int i = 0; i < P.nkeys; ++i)
    dense[i] = ((P.key_src[i] * nd + P.key_dx[i] + P.dmax) * nd + P.key_dy[i] + P.dmax) * nb *
                   nb +
               P.key_b3[i] * nb + P.key_b4[i];
  std::vector<int> rowp;
  std::vector<int4> terms;
  for (int t = 0; t < 3; ++t) {
    c->term_off[t] = (int)terms.size();
    for (int v : P.row_ptr[t]) rowp.push_back(v);
    for (size_t i = 0; i < P.term_key[t].size(); ++i)
      terms.push_back(make_int4(dense[P.term_key[t][i]], P.term_dx[t][i] + P.dmax,
                                P.term_dy[t][i] + P.dmax, (int)P.term_sign[t][i]));
  }
  c->n_terms = (int)terms.size();
  std::vector<int4> gslot = P.gslot;
  for (int4& g : gslot)
    if (g.y >= 0) g.y = dense[g.y];
  TUFRG_CHECK(upload(&c->d_row_ptr, rowp, st));
  TUFRG_CHECK(upload(&c->d_terms, terms, st));
  TUFRG_CHECK(upload(&c->d_gslot, gslot, st));
  // e^{i l.Y} for every phase position Y and every l = (ix, iy)
  std::vector<double2> yph((size_t)P.gy.size() * c->nl);
  std::vector<float2> yph_f(yph.size());
  for (size_t g = 0; !c->mesh && g < P.gy.size(); ++g) {
    const int dx = P.gy[g].x, dy = P.gy[g].y;
    for (int ix = 0; ix < c->ncx; ++ix)
      for (int iy = 0; iy < c->ncy; ++iy) {
        const double a = M_PI * (double)((2 * ix - c->ncx) * dx) / (2.0 * c->ncx) +
                         M_PI * (double)((2 * iy - c->ncy) * dy) / (2.0 * c->ncy);
        const size_t e = g * c->nl + (size_t)ix * c->ncy + iy;
        yph[e] = make_double2(std::cos(a), std::sin(a));
        yph_f[e] = make_float2((float)yph[e].x, (float)yph[e].y);
      }
  }
  if (c->mesh) {  // e^{i l.Y} at the mesh points, l = -pi + 2 pi j / (nc m)
    const int div = c->ncx * c->mesh_m;
    for (size_t g = 0; g < P.gy.size(); ++g)
      for (int l = 0; l < c->nl; ++l) {
        const int2 j = c->mesh_pts[l];
        const double a = M_PI * (double)((2 * j.x - div) * P.gy[g].x) / (2.0 * div) +
                         M_PI * (double)((2 * j.y - div) * P.gy[g].y) / (2.0 * div);
        const size_t e = g * c->nl + l;
        yph[e] = make_double2(std::cos(a), std::sin(a));
        yph_f[e] = make_float2((float)yph[e].x, (float)yph[e].y);
      }
    TUFRG_CHECK(upload(&c->d_mesh_w, c->mesh_w, st));
    TUFRG_CHECK(upload(&c->d_mesh_pts, c->mesh_pts, st));
    // nl w(l) e^{i l.X} at the key positions X = ((dx - dmax)/2, (dy - dmax)/2)
    // for both weight sets: l.X = pi n / (2 nc m) with an integer n, reduced
    // modulo 4 nc m before the sine and cosine
    const int nd = 2 * P.dmax + 1, nx = nd * nd;
    std::vector<double2> e((size_t)2 * nx * c->nl);
    std::vector<float2> e_f(e.size());
    for (int ws = 0; ws < 2; ++ws)
      for (int x = 0; x < nx; ++x) {
        const int dx = x / nd - P.dmax, dy = x % nd - P.dmax;
        for (int l = 0; l < c->nl; ++l) {
          const int2 j = c->mesh_pts[l];
          long long n = (long long)(2 * j.x - div) * dx + (long long)(2 * j.y - div) * dy;
          n %= 4LL * div;
          const double a = M_PI * (double)n / (2.0 * div);
          const double w = c->mesh_w[(size_t)ws * c->nl + l] * c->nl;
          const size_t o = ((size_t)ws * c->nl + l) * nx + x;  // [2][nl][nd^2]
          e[o] = make_double2(w * std::cos(a), w * std::sin(a));
          e_f[o] = make_float2((float)e[o].x, (float)e[o].y);
        }
      }
    TUFRG_CHECK(upload(&c->d_mesh_e, e, st));
    TUFRG_CHECK(upload(&c->d_mesh_e_f, e_f, st));
    if (c->p.precision != TUFRG_FP64) {
      // tensor-core operands of the FP32 quadrature: A [2][mpad][lp] BF16 hi/lo
      // (row 2x: Re, 2x + 1: Im of the phases of position x; zero padding),
      // B [3][npad][lp] packed per right-hand side; splits of the points for
      // about one CTA per SM
      const int lp = (c->nl + 63) / 64 * 64;
      const int mpad = (2 * nx + 127) / 128 * 128;
      const int npad = (c->nff * c->nff + 127) / 128 * 128;
      std::vector<uint16_t> ahi((size_t)2 * mpad * lp, 0), alo(ahi.size(), 0);
      for (int ws = 0; ws < 2; ++ws)
        for (int l = 0; l < c->nl; ++l)
          for (int x = 0; x < nx; ++x) {
            const double2 v = e[((size_t)ws * c->nl + l) * nx + x];
            const double part[2] = {v.x, v.y};
            for (int q = 0; q < 2; ++q) {
              const float f = (float)part[q];
              const uint16_t h = bf16_rne(f);
              const size_t o = ((size_t)ws * mpad + 2 * x + q) * lp + l;
              ahi[o] = h;
              alo[o] = bf16_rne(f - bf16_value(h));
            }
          }
      uint16_t *dah = nullptr, *dal = nullptr, *dbh = nullptr, *dbl = nullptr;
      TUFRG_CHECK(upload(&dah, ahi, st));
      c->d_mesh_ahi = dah;
      TUFRG_CHECK(upload(&dal, alo, st));
      c->d_mesh_alo = dal;
      TUFRG_CHECK(alloc(&dbh, (size_t)3 * npad * lp));
      c->d_mesh_bhi = dbh;
      TUFRG_CHECK(alloc(&dbl, (size_t)3 * npad * lp));
      c->d_mesh_blo = dbl;
      const int tiles = 3 * (mpad / 128) * (npad / 128), nkb = lp / 64;
      int kz = std::max(1, std::min(nkb, sm_count() / tiles));
      c->mesh_kbs = (nkb + kz - 1) / kz;
      c->mesh_kz = (nkb + c->mesh_kbs - 1) / c->mesh_kbs;
      c->mesh_lp = lp;
      c->mesh_mpad = mpad;
      c->mesh_npad = npad;
    }
    // chunks of mesh points for at most one wave of partial-sum CTAs at two
    // CTAs per SM (the FP32 kernel's residency)
    const int tiles = 3 * ((c->nff * c->nff + kMeshAB - 1) / kMeshAB);
    int chunks = std::max(1, 2 * sm_count() / tiles);
    int lc = (c->nl + chunks - 1) / chunks;
    lc = (lc + 31) / 32 * 32;
    c->mesh_lc = lc;
    c->mesh_chunks = (c->nl + lc - 1) / lc;
  }
  TUFRG_CHECK(upload(&c->d_yphase, yph, st));
  TUFRG_CHECK(upload(&c->d_yphase_f, yph_f, st));
  return TUFRG_OK;
}

void free_device(tufrg_ctx* c) {
  free_refinement(c);
  flow_drop_graphs(c);
  free_flow(c);
  view_free(c->view);
  void* own[] = {c->d_ext,     c->d_xiext, c->d_err, c->d_tab, c->d_lambda, c->d_partial,
                 c->d_chi,     c->d_V,     c->d_bt,  c->d_fkey, c->d_y32,
                 c->d_atensor, c->d_par,   c->d_mesh_w, c->d_mesh_pts, c->d_mesh_e,
                 c->d_mesh_e_f, c->d_mesh_ahi, c->d_mesh_alo, c->d_mesh_bhi, c->d_mesh_blo};
  for (void* p : own)
    if (p) cudaFree(p);
  if (!c->borrowed_loops) {
    void* loops[] = {c->d_rowoff,  c->d_kbase,     c->d_Fhi,    c->d_Flo,     c->d_tmap,
                     c->d_rowimg_ptr,
                     c->d_rowimg,  c->d_lrow,      c->d_symperm, c->d_symsign, c->d_kidx,
                     c->d_lgather,
                     c->d_F,       c->d_pairidx,
                     c->d_shift,   c->d_pair,      c->d_acos};
    for (void* p : loops)
      if (p) cudaFree(p);
  }
  if (!c->borrowed_proj) {
    void* proj[] = {c->d_coef,   c->d_phase,   c->d_row_ptr, c->d_terms,
                    c->d_gslot,  c->d_coef_f,  c->d_phase_f, c->d_yphase, c->d_yphase_f};
    for (void* p : proj)
      if (p) cudaFree(p);
  }
  for (cudaEvent_t e : {c->ev_in, c->ev_out, c->ev_fork, c->ev_join, c->ev_stage})
    if (e) cudaEventDestroy(e);
  for (cudaStream_t q : {c->fstream, c->pstream})
    if (q) cudaStreamDestroy(q);
}

}  // namespace tufrg
