// Internal declarations of the TUfRG GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tufrg.h"

#define TUFRG_CUDA(expr)                                      \
  do {                                                        \
    cudaError_t tufrg_e_ = (expr);                            \
    if (tufrg_e_ != cudaSuccess) return tufrg_cuda_fail(tufrg_e_); \
  } while (0)

#define TUFRG_CHECK(expr)                     \
  do {                                        \
    tufrg_status tufrg_s_ = (expr);           \
    if (tufrg_s_ != TUFRG_OK) return tufrg_s_; \
  } while (0)

tufrg_status tufrg_cuda_fail(cudaError_t e);

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
};

struct FlowState;

}  // namespace tufrg

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
  int nrow = 0;                    // l-representative rows (one per pair {l, -l})
  int2* d_shift = nullptr;         // [nrow] l/2 of each row in fine-grid steps
  int2* d_rowmap = nullptr;        // [nrow] (l, partner l) written by each row
  int* d_pair = nullptr;           // [mpad] m*nff+n (or -1)
  double2* d_coef = nullptr;       // [nff][nb] bond coefficients
  double2* d_phase = nullptr;      // [ncx + ncy][2*dmax+1] e^{i l d pi/(2nc)} tables
  int4* d_key = nullptr;           // [nkeys] (src, b3*nb+b4, dx, dy)
  int* d_row_ptr = nullptr;        // [3][nb*nb+1]
  int4* d_terms = nullptr;         // [total terms] (key, dx, dy, sign)
  int term_off[3] = {0, 0, 0};

  // tensor-core loop path (precision BF16X3 / 3XTF32)
  int tc_npad = 0, tc_kpad = 0, tc_kbps = 0, tc_ksplit = 0, tc_nrow_pad = 0, tc_tmem_cols = 0;
  int tc_nsets = 1;                // accumulator sets per channel in TMEM
  int loop_prec = TUFRG_FP64;      // precision of the flow's next loop contractions
  int tc_hx = 0, tc_hy = 0, tc_wy = 0;  // halo of the extended table, its row width
  float4* d_ext = nullptr;         // [(nfx+2hx)*wy] (xi, A, H, |xi|) in FP32 per scale
  int* d_rowoff = nullptr;         // [nrow] sx * wy + sy
  int* d_kbase = nullptr;          // [tc_kpad] loop point offsets in the halo table
  unsigned char* d_Fhi = nullptr;  // [tc_npad][tc_kpad] high parts of F (bf16 or tf32)
  unsigned char* d_Flo = nullptr;  // [tc_npad][tc_kpad] low parts
  float* d_partial_tc = nullptr;   // [tc_ksplit][2][tc_npad][tc_nrow_pad]
  int* d_err = nullptr;            // device error word (bounded waits that gave up)

  // device: workspace
  double* d_lambda = nullptr;      // scalar scale used by the kernels
  double* d_partial = nullptr;     // [ksplit][2][mpad][nrow] split-K partial sums
  double* d_chi = nullptr;         // [2][nl][nff][nff]
  double* d_V = nullptr;           // [3][nl][nff][nff]
  double2* d_bt = nullptr;         // [3][nb*nb][nl] bond-space propagators
  double2* d_fkey = nullptr;       // [nkeys] Fourier values

  // integrator of tufrg_flow_* (allocated on first use) and the library's own
  // stream: flows run there (graph capture needs a non-legacy stream) and are
  // joined to the caller's stream with events
  tufrg::FlowState* flow = nullptr;
  cudaStream_t fstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;

  size_t state_elems() const { return (size_t)3 * nl * nff * nff; }
};

namespace tufrg {

tufrg_status setup_device(tufrg_ctx* c, cudaStream_t st);
void free_device(tufrg_ctx* c);

// kernels (launchers)
tufrg_status launch_scale_tables(tufrg_ctx* c, cudaStream_t st);
tufrg_status launch_loops_fp64(tufrg_ctx* c, double* chi_out, cudaStream_t st);
// projections and products: FP64 arithmetic when prec == TUFRG_FP64, else FP32
tufrg_status launch_project(tufrg_ctx* c, int prec, const double* y, double* v,
                            cudaStream_t st);
tufrg_status launch_products(tufrg_ctx* c, int prec, const double* v, const double* chi,
                             double* dy, const double* d_scale, cudaStream_t st);
tufrg_status launch_set_scalar(double* d, double value, cudaStream_t st);

// steps i-iii at the scale stored in c->d_lambda with loops in precision prec;
// dy scaled by *d_scale if non-null
tufrg_status rhs_device(tufrg_ctx* c, int prec, const double* y, double* dy,
                        const double* d_scale, cudaStream_t st);

tufrg_status prepare_products(tufrg_ctx* c);
tufrg_status prepare_loops_tc(tufrg_ctx* c);
size_t tc_smem_bytes(int npad);
tufrg_status launch_loops_tc(tufrg_ctx* c, double* chi_out, cudaStream_t st);
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

tufrg_status flow_init(tufrg_ctx* c, const tufrg_flow_opts* o, const double* y0, cudaStream_t st);
tufrg_status flow_step(tufrg_ctx* c, int n_steps, tufrg_result* r, cudaStream_t st);
tufrg_status flow_state(tufrg_ctx* c, double* y_out, tufrg_result* r, cudaStream_t st);
void free_flow(tufrg_ctx* c);

}  // namespace tufrg
