// Multi-point views: the per-point descriptors of n contexts, the CTA prefix
// tables of the multi-point launches, and the work items of the persistent
// tensor-core loop kernel.
//
// Work items are (point, tile of l-rows, first K-block, K-blocks); a point's
// rows are spread evenly over ceil(nrow / 128) tiles.  A
// point's loop sum over its nkb K-blocks is cut into ksplit = ceil(nkb/kbps)
// ranges; each range of each tile is one item whose FP32 partial sum is
// combined with the others (fixed order, compensated FP32 pairs, FP64
// result) by the reduction kernel.
// The persistent CTAs take items from a queue ordered by estimated cost,
// longest first, so the uneven points of a batch end together; the tiles of
// one K range stay next to each other in the queue, so that F is read from
// HBM about once however many tiles a point has.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace tufrg {
namespace {

template <class T>
tufrg_status upload_to(T** dptr, const std::vector<T>& h, cudaStream_t st) {
  if (*dptr) cudaFree(*dptr);
  *dptr = nullptr;
  const size_t bytes = std::max<size_t>(h.size(), 1) * sizeof(T);
  if (cudaMalloc((void**)dptr, bytes) != cudaSuccess) return TUFRG_ERR_OOM;
  if (!h.empty())
    TUFRG_CUDA(cudaMemcpyAsync(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return TUFRG_OK;
}

// accumulation chains of at most 5120 (BF16x3) or 4096 (3xTF32, twice the
// MMA instructions per loop point) loop points per item: the tensor core
// rounds the FP32 accumulator once per MMA instruction, so the relative error
// of an item's partial sum grows with its number of K-blocks per
// accumulator set (BF16x3 at 8192 points per item reached ~1e-5 at
// production sizes, 4096 keep it near 5e-6).  The large workload's default
// then takes two items of 72 K-blocks per CTA instead of three of 48
// (323.6 instead of 333 us per launch: one item change less per CTA).
}  // namespace

int max_kbps(int prec) { return (prec == TUFRG_BF16X3 ? 5120 : 4096) / tc_k_per_block(prec); }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    return 1;
  return n;
}

int smem_optin() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 48 * 1024;
  return n;
}

int view_default_kbps(const MultiView& v) {
  if (v.tc_prec == TUFRG_FP64) return 0;
  long long work = 0;  // K-block x tile units
  for (const PointDesc& d : v.h) work += (long long)d.nkb * ((d.row_hi - d.row_lo + 127) / 128);
  const long long S = sm_count(), cap = max_kbps(v.tc_prec);
  const long long waves = std::max(1LL, (work + S * cap - 1) / (S * cap));
  const long long kbps = (work + S * waves - 1) / (S * waves);
  return (int)std::max(1LL, std::min(cap, kbps));
}

tufrg_status view_set_kbps(MultiView& v, int kbps, cudaStream_t st) {
  if (v.tc_prec == TUFRG_FP64) return TUFRG_OK;
  if (kbps < 1 || kbps > max_kbps(v.tc_prec)) return TUFRG_ERR_ARG;
  v.kbps = kbps;
  struct Item {
    int4 it;
    long long cost;  // of the item's K range over all tiles of its point
  };
  std::vector<Item> items;
  size_t off = 0;
  v.npad_max = 16;
  v.tmem_cols = 32;
  for (int i = 0; i < v.n; ++i) {
    PointDesc& d = v.h[i];
    d.ksplit = (d.nkb + kbps - 1) / kbps;
    d.off_partial = (long long)off;
    off += (size_t)d.ksplit * 2 * d.npad * d.nrow_pad;
    v.npad_max = std::max(v.npad_max, d.npad);
    int cols = 32;
    while (cols < d.nsets * 2 * d.npad) cols *= 2;
    v.tmem_cols = std::max(v.tmem_cols, cols);
    const int nr = d.row_hi - d.row_lo, tiles = (nr + 127) / 128;
    // the tiles of one K range one after the other (and ordered as a group):
    // CTAs running at the same time then read the same F columns, from L2
    // after the first
    for (int sp = 0; sp < d.ksplit; ++sp) {
      const int kb0 = sp * kbps, cnt = std::min(kbps, d.nkb - kb0);
      long long cost = 0;  // producers: ~ valid rows per K-block; tensor cores: ~ pair columns
      for (int t = 0; t < tiles; ++t)
        cost += (long long)cnt * (2 * ((t + 1) * nr / tiles - t * nr / tiles) + d.npad);
      for (int t = 0; t < tiles; ++t) items.push_back({make_int4(i, t, kb0, cnt), cost});
    }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const Item& a, const Item& b) { return a.cost > b.cost; });
  std::vector<int4> packed(items.size());
  for (size_t k = 0; k < items.size(); ++k) packed[k] = items[k].it;
  v.n_items = (int)packed.size();
  TUFRG_CHECK(upload_to(&v.d_items, packed, st));
  if (off > v.partial_elems || !v.d_partial) {
    if (v.d_partial) cudaFree(v.d_partial);
    v.d_partial = nullptr;
    v.partial_elems = 0;
    if (cudaMalloc((void**)&v.d_partial, std::max<size_t>(off, 1) * sizeof(float)) != cudaSuccess)
      return TUFRG_ERR_OOM;
    v.partial_elems = off;
  }
  v.ctas = sm_count();
  TUFRG_CHECK(upload_to(&v.d, v.h, st));
  TUFRG_CHECK(prepare_loops_tc_multi(v));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

tufrg_status view_build(MultiView& v, tufrg_ctx* const* ctx, int n, double* const* lam,
                        const int* const* skip, int* err, int tc_prec, int kbps,
                        cudaStream_t st) {
  view_free(v);
  if (n < 1) return TUFRG_ERR_ARG;
  v.n = n;
  v.h.assign(n, PointDesc{});
  v.d_err = err;
  v.tc_prec = tc_prec;
  v.prefix.assign((size_t)kKinds * (n + 1), 0);
  size_t off_state = 0, off_chi = 0, off_bt = 0, off_fkey = 0, off_rowres = 0, off_wstate = 0;
  const bool tc = tc_prec != TUFRG_FP64;
  // the projection form of the whole view (one launch sequence for all points)
  bool grouped = false;
  for (int i = 0; i < n; ++i) grouped = grouped || ctx[i]->nff >= kGroupedNff || ctx[i]->mesh;
  for (int i = 0; i < n; ++i) v.mesh = v.mesh || ctx[i]->mesh;
  if (v.mesh && n != 1) return TUFRG_ERR_ARG;  // a mesh context is a view of its own
  v.proj_grouped = grouped;
  for (int i = 0; i < n; ++i) {
    const tufrg_ctx* c = ctx[i];
    if (tc && c->p.precision != tc_prec) return TUFRG_ERR_ARG;
    PointDesc& d = v.h[i];
    d.nl = c->nl;
    d.nff = c->nff;
    d.nb = c->nb;
    d.ncx = c->ncx;
    d.ncy = c->ncy;
    d.nd = 2 * c->proj.dmax + 1;
    d.nkeys = c->proj.nkeys;
    d.feedback = c->p.feedback;
    d.U = c->p.U;
    for (int t = 0; t < 3; ++t) d.term_off[t] = c->term_off[t];
    for (int t = 0; t < 4; ++t) d.gy_off[t] = c->proj.gy_off[t];
    d.npair = c->npair;
    d.nrow = c->nrow;
    d.row_lo = c->shard_lo;
    d.row_hi = c->shard_hi;
    d.nfx = c->nfx;
    d.nfy = c->nfy;
    d.hx = c->tc_hx;
    d.hy = c->tc_hy;
    d.wy = c->tc_wy;
    d.n_ext = tc ? (c->nfx + 2 * c->tc_hx) * c->tc_wy : 0;
    d.nkb = c->tc_nkb;
    d.kpad_tc = c->tc_kpad;
    d.nrow_pad = c->tc_nrow_pad;
    d.npad = c->tc_npad;
    d.nsets = c->tc_nsets;
    d.off_state = (long long)off_state;
    d.off_chi = (long long)off_chi;
    d.off_bt = (long long)off_bt;
    d.off_fkey = (long long)off_fkey;
    d.off_wstate = (long long)off_wstate;
    off_wstate += (size_t)3 * c->nrow * c->nff * c->nff;
    off_state += (size_t)3 * c->nl * c->nff * c->nff;
    off_chi += (size_t)2 * c->nl * c->nff * c->nff;
    off_bt += ctx_bt_elems(c);
    off_fkey += fkey_elems(2 * c->proj.dmax + 1, c->nb);
    d.tab = c->d_tab;
    d.ext = c->d_ext;
    d.xiext = c->d_xiext;
    d.kbase = c->d_kbase;
    d.rowoff = c->d_rowoff;
    d.Fhi = c->d_Fhi;
    d.Flo = c->d_Flo;
    d.tmap = c->d_tmap;
    d.rowimg_ptr = c->d_rowimg_ptr;
    d.rowimg = c->d_rowimg;
    d.lrow = c->d_lrow;
    d.lgather = c->d_lgather;
    d.pairidx = c->d_pairidx;
    d.symperm = c->d_symperm;
    d.symsign = c->d_symsign;
    d.off_rowres = (long long)off_rowres;
    off_rowres += (size_t)2 * c->nrow * c->npair;
    d.pair = c->d_pair;
    d.coef = c->d_coef;
    d.phase = c->d_phase;
    d.coef_f = c->d_coef_f;
    d.phase_f = c->d_phase_f;
    d.yphase = c->d_yphase;
    d.yphase_f = c->d_yphase_f;
    d.row_ptr = c->d_row_ptr;
    d.terms = c->d_terms;
    d.gslot = c->d_gslot;
    d.gmaxt = c->proj.gmaxt;
    d.lam = lam[i];
    d.skip = skip ? skip[i] : nullptr;
    d.mesh_w = c->d_mesh_w;
    d.mesh_pts = c->d_mesh_pts;
    d.mesh_div = c->ncx * c->mesh_m;
    d.mesh_e = c->d_mesh_e;
    d.mesh_e_f = c->d_mesh_e_f;
    d.mesh_lc = c->mesh_lc;
    d.mesh_chunks = c->mesh_chunks;
    d.mesh_ahi = c->d_mesh_ahi;
    d.mesh_alo = c->d_mesh_alo;
    d.mesh_bhi = c->d_mesh_bhi;
    d.mesh_blo = c->d_mesh_blo;
    d.mesh_lp = c->mesh_lp;
    d.mesh_mpad = c->mesh_mpad;
    d.mesh_npad = c->mesh_npad;
    d.mesh_kz = c->mesh_kz;
    d.mesh_kbs = c->mesh_kbs;
    const int cnt[kKinds] = {
        tc ? table_ctas(d.n_ext, tc_prec) : 0,
        tc ? tc_rows_ctas(d.npair, d.row_lo, d.row_hi) : 0,
        !d.feedback ? 0
        : c->mesh   ? mesh_partial_ctas(c->mesh_chunks, d.nff)
                    : bond_ctas(d.ncx, d.nff),
        d.feedback ? dft_ctas(d.nd) : 0,
        grouped && d.feedback ? d.gy_off[3] : 0,
        contract_ctas(d.nl, d.nff, grouped),
        d.nl,
        d.nrow,
        contract_ctas(d.nrow, d.nff, grouped),
        d.nrow,
    };
    for (int k = 0; k < kKinds; ++k)
      v.prefix[(size_t)k * (n + 1) + i + 1] = v.prefix[(size_t)k * (n + 1) + i] + cnt[k];
    v.nff_max = std::max(v.nff_max, d.nff);
    v.nb_max = std::max(v.nb_max, d.nb);
    v.nd_max = std::max(v.nd_max, d.nd);
    v.nc_sum_max = std::max(v.nc_sum_max, d.ncx + d.ncy);
    const int nf = d.nff == d.nb ? d.nff : 0;
    v.nf_uniform = i == 0 ? nf : (v.nf_uniform == nf ? nf : 0);
  }
  v.state_elems = off_state;
  v.wstate_elems = off_wstate;
  v.chi_elems = off_chi;
  v.bt_elems = off_bt;
  v.fkey_elems = off_fkey;
  v.rowres_elems = off_rowres;
  if (cudaMalloc((void**)&v.d_rowres, std::max<size_t>(off_rowres, 1) * sizeof(double)) !=
      cudaSuccess)
    return TUFRG_ERR_OOM;
  TUFRG_CHECK(upload_to(&v.d_prefix, v.prefix, st));
  if (cudaMalloc((void**)&v.d_counter, sizeof(int)) != cudaSuccess) return TUFRG_ERR_OOM;
  TUFRG_CHECK(prepare_project_multi(v));
  TUFRG_CHECK(prepare_products_multi(v));
  if (tc) return view_set_kbps(v, kbps > 0 ? kbps : view_default_kbps(v), st);
  TUFRG_CHECK(upload_to(&v.d, v.h, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

void view_free(MultiView& v) {
  void* ptrs[] = {v.d, v.d_prefix, v.d_items, v.d_counter, v.d_partial, v.d_rowres};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  v = MultiView();
}

}  // namespace tufrg
