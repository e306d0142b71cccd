// Internal declarations of the TUfRG GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tufrg.h"

#define TUFRG_CUDA(expr)                                                              \
  do {                                                                                \
    cudaError_t tufrg_e_ = (expr);                                                    \
    if (tufrg_e_ != cudaSuccess) return tufrg_cuda_fail_at(tufrg_e_, __FILE__, __LINE__); \
  } while (0)

#define TUFRG_CHECK(expr)                     \
  do {                                        \
    tufrg_status tufrg_s_ = (expr);           \
    if (tufrg_s_ != TUFRG_OK) return tufrg_s_; \
  } while (0)

tufrg_status tufrg_cuda_fail(cudaError_t e);
// records the failing call's source location for tufrg_last_cuda_error
tufrg_status tufrg_cuda_fail_at(cudaError_t e, const char* file, int line);

namespace tufrg {

// One real form factor written as sum_j coef_j * trig_j(k . R_j), trig = cos or sin.
struct TrigTerm {
  double coef;
  bool is_sin;
  int rx, ry;
};

struct FormFactor {
  int shell;
  int parity;                 // f(-k) = parity f(k)
  std::string irrep;          // A1, B1, B2, A2, E
  std::vector<TrigTerm> terms;
};

// Form-factor basis of complete bond shells 0..n_shells (Sec. 3, footnote).
struct Basis {
  int n_shells = 0;
  int nff = 0;
  int nb = 0;
  std::vector<int> bx, by;                    // bonds in the caller's order
  std::vector<FormFactor> ff;                 // canonical order
  std::vector<std::complex<double>> coef;     // [nff][nb]: f_m(k) = sum_b c e^{i k.R_b}
  int max_component = 0;

  tufrg_status build(int n_bonds, const int32_t* bonds);
  double eval(int m, double kx, double ky) const;
  // representation of C4v on the form factors as signed permutations:
  // f_m(g k) = sign[g][m] f_{perm[g][m]}(k) for the 8 elements g (order of
  // kC4v); false if some element is not a signed permutation
  bool point_group(std::vector<int>& perm, std::vector<int>& sign) const;
};

// Scale-independent projection data of Eqs. (proj_VP/VC/VD) in position
// space: Fourier keys (source channel, bond pair, half-integer position X)
// and, per target channel and output bond pair (b1, b2), the list of terms
// (key, half-integer phase position Y, sign).
struct ProjTables {
  int nkeys = 0;
  int dmax = 0;                              // |2X|, |2Y| components <= dmax
  std::vector<int> key_src, key_b3, key_b4, key_dx, key_dy;
  // per target t: CSR over output pairs b1*nb+b2
  std::vector<int> row_ptr[3];
  std::vector<int> term_key[3], term_dy[3], term_dx[3];
  std::vector<double> term_sign[3];
  // the same terms grouped by phase position: the distinct Y of target t
  // are entries gy_off[t] .. gy_off[t + 1] - 1 of gy = (2Y_x, 2Y_y); the
  // terms of position g fill slots g * gmaxt .. of gslot as (b1*nb+b2, key,
  // sign, 0), ordered by output pair, unused slots (-1, -1, 0, 0)
  int gy_off[4] = {0, 0, 0, 0};
  int gmaxt = 0;
  std::vector<int2> gy;
  std::vector<int4> gslot;
};

struct FlowState;

extern const int kC4v[8][2][2];

// One point (one set of model parameters and grids) as the multi-point
// kernels see it.  A context is a batch of one point; a batch context
// (tufrg_batch) holds many.  Offsets locate the point in packed buffers
// (elements of the buffer's own type).
struct PointDesc {
  int nl, nff, nb, ncx, ncy, nd, nkeys, feedback;
  double U;
  int term_off[3];  // term form: first term of target t
  int gy_off[4];    // grouped form: positions Y of target t are gy_off[t] .. gy_off[t + 1] - 1
  int npair, nrow;
  int row_lo, row_hi;  // the loop rows this view's contraction computes (all: 0, nrow)
  // tensor-core loops
  int nfx, nfy, hx, hy, wy, n_ext, nkb, kpad_tc, nrow_pad, npad, nsets, ksplit;
  long long off_state, off_chi, off_bt, off_fkey, off_partial;
  // offset of the point's wedge state [3][nrow][nff][nff]: the state at the
  // representative l of each loop row (flows of a point-group covariant state)
  long long off_wstate;
  const double4_32a* tab;
  const float* xiext;  // [n_ext] xi over the halo table's points (FP32)
  float4* ext;
  const int* kbase;
  const int* rowoff;
  const unsigned char* Fhi;
  const unsigned char* Flo;
  const void* tmap;       // two TMA tensor maps (F hi, F lo), 128 bytes each
  const int* rowimg_ptr;  // [nrow + 1] CSR of the (l, g) each row serves
  const int2* rowimg;
  const int2* lrow;       // [nl] (row, g) serving each l
  const int* lgather;     // [nl][nff][nff] signed row-loop index + 1 of each entry (0: none)
  const int* pairidx;     // [nff][nff] pair index of {m, n}, -1 if forbidden
  const int* symperm;     // [8][nff] signed permutations R^g
  const int* symsign;
  long long off_rowres;   // offset of the point's [2][nrow][npair] row loops
  const int* pair;
  const double2* coef;
  const double2* phase;
  const float2* coef_f;   // the same in FP32 (FP32-arithmetic kernels)
  const float2* phase_f;
  const double2* yphase;  // [phase positions Y][nl] e^{i l.Y}
  const float2* yphase_f;
  const int* row_ptr;  // term form: [3][nb*nb+1] CSR over output pairs
  const int4* terms;   //   (key, 2Y_x + dmax, 2Y_y + dmax, sign)
  const int4* gslot;   // grouped form: [positions Y][gmaxt] (b1*nb+b2, key, sign, 0)
  int gmaxt;
  const double* lam;  // [0] scale of the loops, [1] factor applied to dy when scaled
  const int* skip;    // nonzero: the point does no work (finished flow); may be null
  // non-uniform meshes: [2][nl] quadrature weights of mesh_P and mesh_CD and
  // the lattice coordinates of the points (null on the coarse grid)
  const double* mesh_w;
  const int2* mesh_pts;
  int mesh_div;       // nc m: the lattice of the mesh points
  // [2][nl][nd^2] nl w(l) e^{i l.X} of mesh_P and mesh_CD at the key positions
  // X; the key DFT sums mesh points in mesh_chunks chunks of mesh_lc
  const double2* mesh_e;
  const float2* mesh_e_f;
  int mesh_lc, mesh_chunks;
  // FP32 arithmetic on the tensor cores (null: the CUDA-core quadrature):
  // BF16 hi/lo operands A [2][mesh_mpad][mesh_lp] (the phases' real and
  // imaginary parts per position) and B [3][mesh_npad][mesh_lp] (the state,
  // packed per right-hand side); the points in mesh_kz splits of mesh_kbs
  // K-blocks of 64
  const void* mesh_ahi;
  const void* mesh_alo;
  void* mesh_bhi;
  void* mesh_blo;
  int mesh_lp, mesh_mpad, mesh_npad, mesh_kz, mesh_kbs;
};

// kinds of multi-point launches: per point, a fixed number of CTAs
enum : int {
  kKindTable = 0,  // per-scale FP32 halo table
  kKindReduce,     // split-K combination of the tensor-core partial sums
  kKindBond,       // projections: DFT of the state along y at the Fourier positions
                   // (non-uniform meshes: partial quadrature sums over chunks of points)
  kKindDft,        // projections: DFT along x (meshes: the chunks' sum) and bond
                   // space, the keys of a position
  kKindOverlap,    // projections: key sums and basis change per phase position
  kKindContract,   // projections: phase sums over the positions, per l
  kKindProducts,   // V chi V
  kKindExpand,     // row loops -> loops of every l the row serves
  kKindContractRows,  // projections, phase sums: at the representative l of each row only
  kKindProductsRows,  // V chi V at each row's representative l, written to the l it serves
  kKinds
};

struct MultiView {
  int n = 0;
  std::vector<PointDesc> h;
  PointDesc* d = nullptr;
  std::vector<int> prefix;  // [kKinds][n + 1] first CTA of each point, per kind
  int* d_prefix = nullptr;
  int nff_max = 0, nb_max = 0, nd_max = 0, nc_sum_max = 0;
  int nf_uniform = 0;  // Nff = Nb, the same for every point (else 0)
  // projections in the grouped form (some point has Nff >= kGroupedNff, or a
  // non-uniform mesh), else in the term form
  bool proj_grouped = false;
  bool mesh = false;  // the (single) point lives on a non-uniform mesh
  // tensor-core loops: work items (point, l-tile, first K-block, K-blocks)
  // taken from a queue by persistent CTAs
  int tc_prec = TUFRG_FP64;  // TUFRG_FP64: no tensor-core loops
  int kbps = 0, n_items = 0, ctas = 0, npad_max = 0, tmem_cols = 0;
  int4* d_items = nullptr;
  int* d_counter = nullptr;
  float* d_partial = nullptr;
  size_t partial_elems = 0;
  int* d_err = nullptr;  // error word of the bounded waits
  double* d_rowres = nullptr;  // loops of the rows, FP64, all points
  // elements of the packed buffers: state (y, V, dy), loops, bond space, keys
  size_t state_elems = 0, chi_elems = 0, bt_elems = 0, fkey_elems = 0, rowres_elems = 0;
  size_t wstate_elems = 0;
  int total(int kind) const { return prefix[(size_t)kind * (n + 1) + n]; }
  const int* dprefix(int kind) const { return d_prefix + (size_t)kind * (n + 1); }
};

}  // namespace tufrg

struct tufrg_surrogate;

// Opaque context of the C ABI.
struct tufrg_ctx {
  tufrg_params p{};
  std::vector<int32_t> bonds;
  tufrg::Basis basis;
  tufrg::ProjTables proj;

  int ncx = 0, ncy = 0, nl = 0, nfx = 0, nfy = 0, nf = 0, nff = 0, nb = 0;
  int npair = 0, mpad = 0;         // parity-allowed pairs m <= n, padded
  int kdim = 0, kpad = 0;          // half-zone loop points, padded
  int ksplit = 0, kchunk = 0;      // split of the loop sum over CTAs
  int rm = 1, mtiles = 1;          // FP64 loop kernel: pairs per thread, pair tiles
  std::vector<int> pair_m, pair_n;

  // device: scale-independent tables
  double4_32a* d_tab = nullptr;        // [nf] (xi, A, H, 0) -- A, H filled per scale
  int2* d_kidx = nullptr;          // [kpad] fine-grid (ix, iy) of each loop point (-1 pad)
  double* d_F = nullptr;           // [mpad][kpad] weight * f_m f_n / Nf
  int nrow = 0;                    // loop rows (point-group classes of l)
  int shard_lo = 0, shard_hi = 0;  // rows of the loop contraction (all unless sharded)
  bool c4v = false;                // rows serve C4v orbits
  int2* d_shift = nullptr;         // [nrow] l/2 of each row in fine-grid steps
  int* d_rowimg_ptr = nullptr;     // [nrow + 1] CSR over d_rowimg
  int2* d_rowimg = nullptr;        // [nl] (l, g): chi(l) = R^g chi(row) R^g^T
  int2* d_lrow = nullptr;          // [nl] (row, g) serving each l
  int* d_lgather = nullptr;        // [nl][nff][nff] +-(row npair + pair + 1): entry (m, n)
                                   // of l's loops in the row loops, signed; 0: forbidden
  int* d_pairidx = nullptr;        // [nff][nff] index of the pair {m, n} (-1: forbidden)
  int* d_symperm = nullptr;        // [8][nff] R^g as signed permutations:
  int* d_symsign = nullptr;        //   (R^g chi R^g^T)_mn = s_m s_n chi_{p(m) p(n)}
  int* d_pair = nullptr;           // [mpad] m*nff+n (or -1)
  double2* d_coef = nullptr;       // [nff][nb] bond coefficients
  double2* d_phase = nullptr;      // [ncx + ncy][2*dmax+1] e^{i l d pi/(2nc)} tables
  float2* d_coef_f = nullptr;      // d_coef, d_phase rounded to FP32
  float2* d_phase_f = nullptr;
  double2* d_yphase = nullptr;     // [ProjTables::gy][nl] e^{i l.Y}, FP64 and FP32
  float2* d_yphase_f = nullptr;
  int* d_row_ptr = nullptr;        // term form: [3][nb*nb+1]
  int4* d_terms = nullptr;         //   [total terms] (key, dx, dy, sign)
  int term_off[3] = {0, 0, 0};
  int n_terms = 0;                 //   all targets
  int4* d_gslot = nullptr;         // grouped form: ProjTables::gslot
  // precomputed projection tensors (tufrg_atensor_build): three stored
  // pairs and four state vectors in the context's arithmetic type
  void* d_atensor = nullptr;
  bool atensor_ready = false;
  int* d_par = nullptr;            // [nff] parity of each form factor
  // Fermi-surface refinement of the loop cells (tufrg_set_refinement): s x s
  // sub-points (s = 1: off), band kappa Lambda, active below Lambda_on;
  // dispersion on the half-cell grid (FP64), dispersion and form factors on
  // the sub-point grid (arithmetic type), the bond vectors
  int ref_s = 1;
  double ref_kappa = 0.0, ref_lam_on = 0.0;
  void* d_ref_xi2 = nullptr;
  void* d_ref_xis = nullptr;
  void* d_ref_ffs = nullptr;
  int* d_ref_bonds = nullptr;
  void* d_ref_part = nullptr;  // [nseg][2][rows][npair] the row segments' sums
  // analytic-xi mode (nf not a multiple of 2 nc, FP64 loops): per loop row the
  // cosines of p +- l/2 per direction, [nrow][2 nfx + 2 nfy]
  bool analytic = false;
  double* d_acos = nullptr;
  int ref_nseg = 1, ref_klen = 0;
  // non-uniform bosonic meshes (tufrg_setup_mesh): the l are mesh points
  // l = -pi + 2 pi j / (nc m) of the union of mesh_P and mesh_CD, with each
  // channel's quadrature weights (zero off its mesh)
  bool mesh = false;
  int mesh_m = 1;
  std::vector<int2> mesh_pts;
  std::vector<double> mesh_w;      // [2][nl]: weights of mesh_P, of mesh_CD
  double* d_mesh_w = nullptr;
  int2* d_mesh_pts = nullptr;
  double2* d_mesh_e = nullptr;  // [2][nl][nd^2] nl w e^{i l.X} (FP64, FP32 copy)
  float2* d_mesh_e_f = nullptr;
  int mesh_lc = 0, mesh_chunks = 0;
  // tensor-core quadrature operands (FP32-arithmetic contexts)
  void* d_mesh_ahi = nullptr;
  void* d_mesh_alo = nullptr;
  void* d_mesh_bhi = nullptr;
  void* d_mesh_blo = nullptr;
  int mesh_lp = 0, mesh_mpad = 0, mesh_npad = 0, mesh_kz = 0, mesh_kbs = 0;

  // tensor-core loop path (precision BF16X3 / 3XTF32)
  int tc_npad = 0, tc_kpad = 0, tc_nkb = 0, tc_nrow_pad = 0;
  int tc_nsets = 1;                // accumulator sets per channel in TMEM
  int loop_prec = TUFRG_FP64;      // precision of the flow's next loop contractions
  int tc_hx = 0, tc_hy = 0, tc_wy = 0;  // halo of the extended table, its row width
  float4* d_ext = nullptr;         // halo table over [(nfx+2hx)*wy] points, FP32 per scale:
                                   // A = 1/(Omega+|xi|), xi (BF16X3: pair layout)
  float* d_xiext = nullptr;        // [(nfx+2hx)*wy] xi at the halo table's points, FP32
  int* d_rowoff = nullptr;         // [nrow] sx * wy + sy
  int* d_kbase = nullptr;          // [tc_kpad] loop point offsets in the halo table
  unsigned char* d_Fhi = nullptr;  // [tc_npad][tc_kpad] high parts of F (bf16 or tf32)
  unsigned char* d_Flo = nullptr;  // [tc_npad][tc_kpad] low parts
  void* d_tmap = nullptr;          // TMA tensor maps of d_Fhi, d_Flo (2 x 128 bytes)
  int* d_err = nullptr;            // device error word (bounded waits that gave up)

  // device: workspace
  double* d_lambda = nullptr;      // scalar scale used by the kernels
  double* d_partial = nullptr;     // [ksplit][2][mpad][nrow] split-K partial sums
  double* d_chi = nullptr;         // [2][nl][nff][nff]
  double* d_V = nullptr;           // [3][nl][nff][nff] (FP32 couplings in its first half)
  float* d_y32 = nullptr;          // FP32 copy of a state (mixed-precision contexts)
  double2* d_bt = nullptr;         // the state's DFT along y, then the overlap sums
                                   // H [positions Y][nff][nff] (bt_region)
  double2* d_fkey = nullptr;       // Fourier values of the keys, dense (fkey_elems)

  // integrator of tufrg_flow_* (allocated on first use) and the library's own
  // stream: flows run there (graph capture needs a non-legacy stream) and are
  // joined to the caller's stream with events
  tufrg::FlowState* flow = nullptr;
  tufrg::MultiView view;           // this context as a batch of one point
  bool borrowed_loops = false;     // loop / projection tables owned by another context
  bool borrowed_proj = false;
  tufrg_surrogate* sur = nullptr;  // loop surrogate of the flows (tufrg_surrogate_attach)
  int sur_every = 8;               // accepted steps between exact judgements
  double sur_tol = 1e-3;           // largest accepted relative error of its loops
  cudaStream_t fstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // tufrg_rhs: the right-hand side captured as a graph per (y, dy) pair it
  // was called with, for the last kRhsGraphs pairs (a caller cycling through
  // a few buffer pairs replays their graphs; launched on fstream after the
  // scale is set)
  static constexpr int kRhsGraphs = 4;
  struct RhsGraph {
    cudaGraphExec_t exec = nullptr;
    const double* y = nullptr;
    double* dy = nullptr;
    unsigned long long used = 0;  // call count at the last use
  };
  RhsGraph rhs_graphs[kRhsGraphs];
  unsigned long long rhs_calls = 0;
  // the projections of a right-hand side run on their own stream, beside the
  // loop contraction (fork after the stage combination, join before the
  // products; branches of the captured flow graphs)
  cudaStream_t pstream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_stage = nullptr;  // flows: the stage combination joins the projection stream

  size_t state_elems() const { return (size_t)3 * nl * nff * nff; }
};

namespace tufrg {

// Tables a new context may take over from an existing one instead of
// building them: loops (same fine and coarse grids, bonds, precision) and
// projections (same coarse grid and bonds).  own_view: build the context's
// batch-of-one view (contexts made for a tufrg_batch skip it).
// workspace: allocate the context's own right-hand-side workspace, stream
// and events (batch points use the batch's).
// A non-uniform mesh: refinement factor m, lattice points and the
// quadrature weights of mesh_P and mesh_CD ([2][points]).
struct MeshSpec {
  int m = 1;
  std::vector<int2> pts;
  std::vector<double> w;
};
struct SetupShare {
  const tufrg_ctx* loops = nullptr;
  const tufrg_ctx* proj = nullptr;
  bool own_view = true;
  bool workspace = true;
  const MeshSpec* mesh = nullptr;  // the context's l are this mesh's points
};
tufrg_status setup_device(tufrg_ctx* c, cudaStream_t st, const SetupShare& share = SetupShare());
// validation, basis and setup_device (tufrg_setup with shared tables)
tufrg_status create_context(const tufrg_params* p, cudaStream_t st, const SetupShare& share,
                            tufrg_ctx** out);
// drops the captured flow graphs (after a change of the tensor-core work items)
// drops the captured graphs (flow attempts, tufrg_rhs) after a change of
// the launch configuration (autotuning, surrogate)
void flow_drop_graphs(tufrg_ctx* c);

// loop "precision" of a flow whose loops the attached surrogate gives
constexpr int kLoopSurrogate = 3;
// the surrogate's loops of every l at the scale in c->d_lambda (forbidden
// pairs untouched); its work buffers must exist before a graph capture (the
// first call makes them)
tufrg_status surrogate_loops(tufrg_surrogate* s, tufrg_ctx* c, double* chi, cudaStream_t st);
// relative max-norm error of the surrogate's loops against the exact ones in
// precision exact_prec, at the scale in c->d_lambda (blocks; leaves the
// surrogate's loops in c->d_chi)
tufrg_status surrogate_judge(tufrg_surrogate* s, tufrg_ctx* c, int exact_prec, double* rel,
                             cudaStream_t st);
// times candidate work-item sizes of the view's tensor-core loops; run sets
// the scale(s) the view's points read and launches the contraction once
tufrg_status autotune_view(MultiView& v, tufrg_status (*run)(void*, cudaStream_t), void* arg,
                           tufrg_tune_report* rep, cudaStream_t st);
void free_device(tufrg_ctx* c);

// kernels (launchers)
tufrg_status launch_scale_tables(tufrg_ctx* c, cudaStream_t st);
tufrg_status launch_loops_fp64(tufrg_ctx* c, double* chi_out, cudaStream_t st);
tufrg_status launch_loops_fp64_rows(tufrg_ctx* c, cudaStream_t st, cudaEvent_t* ev = nullptr);
// projections and products: FP64 arithmetic when prec == TUFRG_FP64, else FP32
tufrg_status launch_set_scalar(double* d, double value, cudaStream_t st);

// steps i-iii at the scale stored in c->d_lambda with loops in precision prec;
// dy scaled by c->d_lambda[1] if scaled
// wedge: y and dy in the wedge layout [3][nrow][nff][nff] of a point-group
// covariant state (flows), projections and products at the rows'
// representative l only
// y32: an FP32 copy of y already on the way (made by the caller on c->pstream,
// before the call), or null
tufrg_status rhs_device(tufrg_ctx* c, int prec, const double* y, double* dy, bool scaled,
                        cudaStream_t st, bool wedge = false, const float* y32 = nullptr);
// arithmetic of the projections and products for loops in precision prec:
// FP64 for an FP64 context and for FP64 loops, else FP32
int rhs_arith(const tufrg_ctx* c, int prec);
// element-wise copies FP64 -> FP32 (rounded to nearest) and FP32 -> FP64
tufrg_status launch_to_f32(const double* x, float* y, size_t n, cudaStream_t st);
tufrg_status launch_to_f64(const float* x, double* y, size_t n, cudaStream_t st);

// multi-point views (multi.cpp): descriptors of n contexts packed one after
// the other; lam[i], skip[i] are per-point device pointers (skip may be null)
tufrg_status view_build(MultiView& v, tufrg_ctx* const* ctx, int n, double* const* lam,
                        const int* const* skip, int* err, int tc_prec, int kbps,
                        cudaStream_t st);
tufrg_status view_set_kbps(MultiView& v, int kbps, cudaStream_t st);
int view_default_kbps(const MultiView& v);
void view_free(MultiView& v);
int sm_count();
// the largest dynamic shared memory a CTA may opt in to on the current device
// (the attribute is per function and process-wide: kernels shared by
// contexts of different sizes get the device limit once, never a
// context's own size, which a later, smaller context would lower)
int smem_optin();

// tensor-core loops of every point (zero: clear chi first; the kernels write
// only the parity-allowed pairs)
tufrg_status launch_loops_tc_multi(const MultiView& v, double* chi, cudaStream_t st);
// loops of every l from the row loops in v.d_rowres (writes every entry)
tufrg_status launch_expand_multi(const MultiView& v, double* chi, cudaStream_t st);
// split-K combinations into the row loops (tensor-core partials of every
// point of v; FP64 partials of one context)
int rows_reduce_ctas(int npair, int nrow);
int tc_rows_ctas(int npair, int row_lo, int row_hi);
tufrg_status launch_tc_rows_multi(const MultiView& v, cudaStream_t st);
tufrg_status launch_fp64_rows(const double* partial, int mpad, int ksplit, int npair, int nrow,
                              double* rowres, cudaStream_t st);
size_t tc_smem_bytes(int npad);
// TMA tensor maps of a context's F parts into c->d_tmap
tufrg_status make_f_tensor_maps(tufrg_ctx* c, cudaStream_t st);
int tc_k_per_block(int prec);
// the most K-blocks one work item accumulates in one FP32 chain
int max_kbps(int prec);
int table_ctas(int n_ext, int prec);
tufrg_status prepare_loops_tc_multi(const MultiView& v);
tufrg_status prepare_project_multi(const MultiView& v);
tufrg_status prepare_products_multi(const MultiView& v);
int bond_ctas(int ncx, int nff);
int dft_ctas(int nd);
// Fourier values of the keys, numbered densely over (source, 2X_x, 2X_y, b3, b4)
size_t fkey_elems(int nd, int nb);
int contract_ctas(int nl, int nff, bool grouped);
// the projections of a view take the grouped form from this form-factor count on
constexpr int kGroupedNff = 21;
// the largest form-factor count the kernels accept (complete shells up to 29)
constexpr int kMaxNf = 32;
// elements of a point's projection workspace: the state's DFT along y
// [3][ncx][nd][nff*nff], later reused for the overlap sums [positions Y][nff][nff]
size_t bt_region(int ncx, int nd, int nff, int ny_total);
// mesh key DFT: CTAs of the partial sums over chunks of mesh points, and the
// partial sums' elements [3][chunks][nd^2][nff^2] (complex; in the bt region)
constexpr int kMeshAB = 64;  // entries (a, b) per CTA of the partial sums
int mesh_partial_ctas(int chunks, int nff);
size_t mesh_partial_elems(int chunks, int nd, int nff);
// projection workspace of a context (complex elements)
size_t ctx_bt_elems(const tufrg_ctx* c);
// tensor-core quadrature of the mesh key DFT (FP32 arithmetic): packs the
// state (wedge: from the rows' representatives) and writes the FP32 partial
// products [3][kz][mpad][npad] to part
tufrg_status prepare_mesh_tc();
tufrg_status launch_mesh_tc(const PointDesc& d, const float* y, bool wedge, float* part, int* err,
                            cudaStream_t st);
// projections and products of every point; bt, fkey: packed workspaces.
// rows: the state in the wedge layout (a point-group covariant state at the
// representative l of each loop row), the projected couplings at the
// representatives, in the wedge layout
// y and out hold doubles for prec == TUFRG_FP64, else floats (FP32 arithmetic)
tufrg_status launch_project_multi(const MultiView& v, int prec, const void* y, void* out,
                                  void* bt, void* fkey, cudaStream_t st, bool rows = false);
// chi == nullptr: the loops of each l are gathered from the row loops
// v.d_rowres (the orbit expansion fused into the products).  rows (with chi
// == nullptr): couplings and dy in the wedge layout, the products at each
// row's representative l only (a covariant state's right-hand side)
// vin: the couplings, doubles for prec == TUFRG_FP64, else floats
tufrg_status launch_products_multi(const MultiView& v, int prec, const void* vin,
                                   const double* chi, double* dy, bool scaled, cudaStream_t st,
                                   bool rows = false);
// largest |y(g l) - R^g y(l) R^g^T| over every l a row serves (l the row's
// representative) and largest |y|, for each point of the view, into dev[2 * i],
// dev[2 * i + 1] as the bit patterns of non-negative doubles
tufrg_status launch_covariance_check(const MultiView& v, const double* y,
                                     unsigned long long* dev, cudaStream_t st);
// the wedge layout [3][nrow][nff][nff] of each point's state (its values at
// the rows' representatives) from the full state, and back: expand writes
// every l a row serves as y(g l) = R^g y(l) R^g^T
tufrg_status launch_wedge_compress(const MultiView& v, const double* y, double* w,
                                   cudaStream_t st);
tufrg_status launch_wedge_expand(const MultiView& v, const double* w, double* y,
                                 cudaStream_t st);
// loop contraction up to the row loops in c->view.d_rowres (no expansion);
// prec must not be the surrogate
tufrg_status launch_loop_rows(tufrg_ctx* c, int prec, cudaStream_t st);
// ev (optional): events recorded just before and after the contraction
// kernel itself, on its stream
tufrg_status launch_loops_tc_rows_multi(const MultiView& v, cudaStream_t st,
                                        cudaEvent_t* ev = nullptr);
// loops in the given precision (the context's, or FP64)
tufrg_status launch_loops(tufrg_ctx* c, int prec, double* chi_out, cudaStream_t st);

// The FP64 loop contraction on explicitly given buffers (same kernels and
// layouts as launch_loops_fp64, without a context).
struct LoopBuffers {
  double4_32a* tab;
  const int2* kidx;
  const double* F;
  const int2* shift;
  const int2* rowmap;
  const double* lambda;
  const int* pair;
  double* partial;
  int nf, nfx, nfy, nl, nrow, nff, npair, mpad, kpad, kchunk, ksplit, mtiles, rm;
};
tufrg_status launch_loops_fp64_buffers(const LoopBuffers& b, double* chi, cudaStream_t st);

// Fermi-surface refinement of the loop cells: tables for (s, kappa,
// Lambda_on) (s = 1, kappa = 0 or Lambda_on = 0: off), the correction of the
// row loops of the rows the context computes (after their combination), and
// release of the tables
tufrg_status set_refinement(tufrg_ctx* c, int s, double kappa, double lam_on, cudaStream_t st);
tufrg_status launch_refine_rows(tufrg_ctx* c, cudaStream_t st);
void free_refinement(tufrg_ctx* c);

// precomputed projection tensors: bytes they take (TUFRG_ERR_ARG when the
// basis is too large), their construction, and V from them
tufrg_status atensor_bytes(const tufrg_ctx* c, size_t* bytes);
tufrg_status atensor_build(tufrg_ctx* c, cudaStream_t st);
tufrg_status atensor_project(tufrg_ctx* c, const double* y, double* v, cudaStream_t st);

tufrg_status flow_init(tufrg_ctx* c, const tufrg_flow_opts* o, const double* y0, cudaStream_t st);
tufrg_status flow_step(tufrg_ctx* c, int n_steps, tufrg_result* r, cudaStream_t st);
tufrg_status flow_state(tufrg_ctx* c, double* y_out, tufrg_result* r, cudaStream_t st);
void free_flow(tufrg_ctx* c);

}  // namespace tufrg
