/*
 * tufrg.h -- C ABI of the GB300 TUfRG right-hand-side library.
 *
 * The library computes the right-hand side of the Lambda-flow of the
 * truncated-unity fRG (Lichtenstein et al., arXiv:1604.06296) for the
 * exchange propagators P, C, D of the t-t' Hubbard model on the square
 * lattice in a bond form-factor basis, and integrates that flow.
 *
 * Conventions shared by every call
 *  - Energies are in units of the hopping t (any t > 0 is accepted).
 *  - Momentum grids: n points per direction at k_i = -pi + 2 pi i / n.
 *    The coarse (bosonic, "l") grid has Nl = nc_x * nc_y points, index
 *    l = ix * nc_y + iy.  The fine loop grid has nf_x * nf_y points.
 *  - Form factors: the library builds Nff real orthonormal C4v-adapted
 *    functions from the bond list (Sec. 3).  Their order is canonical:
 *    shell by shell; within a shell A1, then B1/B2/A2, then E pairs
 *    (x-like, y-like), in the order
 *      shell 0: 1
 *      shell 1: cx+cy, cx-cy, r2 sx, r2 sy
 *      shell 2: 2cxcy, 2sxsy, 2sxcy, 2cxsy
 *      shell 3: c2x+c2y, c2x-c2y, r2 s2x, r2 s2y
 *      shell 4: r2(c2x cy+cx c2y), r2(c2x cy-cx c2y), r2(s2x sy+sx s2y),
 *               r2(s2x sy-sx s2y), 2 s2x cy, 2 cx s2y, 2 sx c2y, 2 c2x sy
 *      shell 5: 2c2xc2y, 2s2xs2y, 2s2xc2y, 2c2xs2y
 *      shell 6: c3x+c3y, c3x-c3y, r2 s3x, r2 s3y
 *    (c = cos, s = sin, r2 = sqrt 2, arguments k_x, k_y).
 *  - State layout: y = (P, C, D) as double [3][Nl][Nff][Nff], row-major.
 *    Loops: double [2][Nl][Nff][Nff] (pp, ph).  Projected couplings:
 *    double [3][Nl][Nff][Nff] (V^P, V^C, V^D).
 *  - Pointers named *_dev are device pointers owned by the caller (e.g.
 *    allocated by torch); the library never frees them.  Host pointers are
 *    read during the call only.
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream).  All
 *    device work of a call is ordered on that stream; calls return once the
 *    work is enqueued, except tufrg_flow (returns when the flow finished).
 *  - Every call returns a tufrg_status and never aborts the process.  An
 *    invalid argument returns TUFRG_ERR_ARG before any device work.  A CUDA
 *    error returns TUFRG_ERR_CUDA; errors of asynchronous work can surface
 *    at a later call on the same stream.
 *  - Readings of the paper the results depend on: the Omega-cutoff
 *    propagator G = k0^2/(k0^2 + Omega^2) / (i k0 - xi_k) at T = 0 with the
 *    frequency integral done in closed form; loops at bosonic frequency 0;
 *    every bosonic momentum is folded into [-pi, pi)^2 and the half momenta
 *    l/2 are formed from that representative; the k, k' integrals of the
 *    projections are averages over the coarse grid; V0 = U on site.
 */
#ifndef TUFRG_H
#define TUFRG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tufrg_ctx tufrg_ctx;

typedef enum {
  TUFRG_OK = 0,
  TUFRG_ERR_ARG = -1,            /* invalid argument or unsupported size */
  TUFRG_ERR_CUDA = -2,           /* a CUDA runtime call or launch failed */
  TUFRG_ERR_NONFINITE = -3,      /* NaN/Inf in the state during a flow */
  TUFRG_ERR_STEP_UNDERFLOW = -4, /* adaptive step fell below 1e-12 in ln Lambda */
  TUFRG_ERR_TIMEOUT = -5,        /* a bounded device wait gave up */
  TUFRG_ERR_OOM = -6,            /* device allocation failed */
  TUFRG_ERR_STATE = -7           /* call out of order (e.g. a step before tufrg_flow_init) */
} tufrg_status;

typedef enum {
  TUFRG_FP64 = 0,    /* everything in FP64 (loops on DFMA) */
  TUFRG_3XTF32 = 1,  /* loops on tcgen05, kind::tf32, hi/lo split, 3 products, FP32
                        accumulation; projections and products in FP32 arithmetic;
                        state, derivative, step control in FP64 */
  TUFRG_BF16X3 = 2   /* as 3XTF32 with kind::f16 (bf16) hi/lo operands */
} tufrg_precision;

typedef enum {
  TUFRG_DOPRI5 = 0,  /* adaptive Dormand-Prince 5(4) in s = ln Lambda */
  TUFRG_RK4 = 1      /* classic RK4, fixed step h0 in s = ln Lambda */
} tufrg_method;

/* Model and discretisation of one phase-diagram point. */
typedef struct {
  int32_t lattice;        /* 0 = square lattice (the only one supported) */
  double t, tp, mu, U;    /* hoppings t, t' (Eq. hubb-disp), chemical potential,
                             on-site U (bare V0 = U) */
  int32_t n_bonds;        /* bond list: lattice vectors (x, y), host memory */
  const int32_t* bonds;   /* [n_bonds][2]; must be complete shells 0..n, n <= 6 */
  int32_t nc_x, nc_y;     /* coarse grid; even, >= 2*max|R|+1 */
  int32_t nf_x, nf_y;     /* fine grid; nf % 4 == 0; nf % (2 nc) == 0 puts p +- l/2
                             on the fine grid (table mode, every precision); other
                             grids run in the analytic-xi mode, FP64 loops only:
                             xi(p +- l/2) from per-row cosine tables (Sec. 3,
                             Eq. hubb-disp), no refinement (TUFRG_ERR_STATE) */
  int32_t precision;      /* tufrg_precision of the loop contraction */
  int32_t feedback;       /* 1 = full inter-channel projections (Eqs. proj_VP..VD);
                             0 = projections off: V^P = V0 - P, V^C = V0 + C,
                             V^D = V0 + D (single-channel ladders) */
} tufrg_params;

/* Options of tufrg_flow. */
typedef struct {
  double lambda0;         /* initial scale (> lambda_min) */
  double lambda_min;      /* final scale if no divergence */
  double threshold;       /* stop when max |B_mn(l)|, B in {P,C,D}, exceeds it */
  double rtol, atol;      /* DoPri5 error control (max norm) */
  double h0;              /* initial (DoPri5) or fixed (RK4) step |h| in ln Lambda */
  int32_t method;         /* tufrg_method */
  int32_t max_steps;      /* tufrg_flow: step budget (accepted + rejected attempts) */
  int32_t n_checkpoints;  /* dense output at these scales (host array, any order) */
  const double* checkpoints;
  double* checkpoint_states_dev; /* [n_checkpoints][3][Nl][Nff][Nff]; entries of
                                    scales not reached are left untouched; must stay
                                    valid until the flow has finished */
  double fp64_above;      /* > 0: once an accepted step has max |B| above this, the
                             loops of the remaining steps run in FP64 (a context set up
                             with a tensor-core precision only); 0: never switch */
} tufrg_flow_opts;

/* Result of tufrg_flow / tufrg_flow_step / tufrg_flow_state. */
typedef struct {
  double lambda_c;        /* critical scale if diverged, else the scale reached */
  double h_next;          /* size |h| in ln Lambda of the next step attempt */
  int32_t diverged;       /* 1 if the threshold was crossed */
  int32_t finished;       /* 1 if diverged or Lambda_min was reached */
  int32_t channel;        /* 0 = P (pairing), 1 = C (magnetic), 2 = D (charge) */
  int32_t l_index, m, n;  /* location of max |B| in the state (smallest flat index);
                             filled by tufrg_flow and tufrg_flow_state */
  double max_abs;         /* max |B| of the state (tufrg_flow, tufrg_flow_state) */
  double lambda_switch;   /* scale after which the loops ran in FP64 (0: no switch) */
  int64_t n_rhs, n_accepted, n_rejected;
  /* flows with a loop surrogate attached (tufrg_surrogate_attach): */
  double lambda_surrogate_off; /* scale at which the judge rejected the surrogate
                                  (0: never rejected, or no surrogate) */
  int64_t n_rhs_surrogate;     /* right-hand sides whose loops the surrogate gave */
  int64_t n_judges;            /* exact-loop judgements made */
} tufrg_result;

/* Sec. 2-4: build the problem (bond basis, grids, dispersion table,
 * scale-independent projection tables, workspace) on the current device.
 * Returns TUFRG_ERR_ARG for an unsupported lattice, incomplete shells, bad
 * grid sizes or precision.  *out receives a context owned by the caller and
 * released by tufrg_destroy.  Blocks until the tables are on the device. */
tufrg_status tufrg_setup(const tufrg_params* p, void* cuda_stream, tufrg_ctx** out);

/* Sec. 4 (the channel meshes): a context whose bosonic momenta are the
 * points of a non-uniform mesh instead of the coarse grid.  The points are
 * host integer pairs points[i][2] = (jx, jy), 0 <= j < nc m, for
 * l = -pi + 2 pi j / (nc m); m is odd (the refinement of a coarse cell into
 * m x m sub-cells), nc_x = nc_y = nc, and nf_x, nf_y are multiples of
 * 2 nc m (l/2 on the fine grid).  w_p[i] and w_cd[i] are the quadrature
 * weights of point i in mesh_P and mesh_CD (zero off that mesh; each set
 * non-negative and summing to one within 1e-9; every point in at least one
 * mesh; no point twice).  The state, couplings, loops and derivative of the
 * context are [3][n_points][Nff][Nff] in the order of the points: the
 * Fourier values of a source channel at the projections' key positions are
 * quadratures over its own mesh (Eqs. proj_VP/VC/VD), the k and k'
 * averages stay those of the coarse grid, and the derivative of P vanishes
 * where w_p = 0, that of C and D where w_cd = 0.  The arrays are copied.
 * Returns TUFRG_ERR_ARG for anything above not met; otherwise as
 * tufrg_setup.  Loop refinement, projection tensors, row sharding and
 * surrogates refuse a mesh context with TUFRG_ERR_STATE. */
tufrg_status tufrg_setup_mesh(const tufrg_params* p, int32_t m, int32_t n_points,
                              const int32_t* points, const double* w_p, const double* w_cd,
                              void* cuda_stream, tufrg_ctx** out);

/* Releases all device and host memory of the context (synchronises). */
void tufrg_destroy(tufrg_ctx* ctx);

/* Sizes: Nl, Nff and the number of bonds.  Any pointer may be NULL. */
tufrg_status tufrg_dims(const tufrg_ctx* ctx, int32_t* nl, int32_t* nff, int32_t* nb);

/* Host evaluation of the form factors that tufrg_setup builds from this
 * bond list (Sec. 3, footnote): out[m * n + i] = f_m(kx[i], ky[i]) for
 * m < Nff (*nff_out receives Nff; out may be NULL to query it).  Host memory
 * only; no device work.  TUFRG_ERR_ARG for an invalid bond list. */
tufrg_status tufrg_eval_formfactors(int32_t n_bonds, const int32_t* bonds, int32_t n,
                                    const double* kx, const double* ky, double* out,
                                    int32_t* nff_out);

/* Step ii, Eq. (chis): scale derivatives of the form-factor projected loops,
 *   chi_dot^pp_mn(l) = d/dLambda (1/Nf) sum_p int dp0/2pi G(l/2+p) G(l/2-p) f_m f_n,
 *   chi_dot^ph_mn(l) = d/dLambda (1/Nf) sum_p int dp0/2pi G(p+l/2) G(p-l/2) f_m f_n,
 * with the Omega-cutoff propagator at T = 0 and Lambda = Omega > 0, in the
 * context's precision.  chi_dot_dev: [2][Nl][Nff][Nff] (pp, ph). */
tufrg_status tufrg_loops(tufrg_ctx* ctx, double lambda, double* chi_dot_dev,
                         void* cuda_stream);

/* Step i, Eqs. (proj_VP/VC/VD): projected couplings V^P, V^C, V^D from the
 * state y = (P, C, D) and the bare U (honours the feedback flag).
 * y_dev: [3][Nl][Nff][Nff]; v_dev: [3][Nl][Nff][Nff]; may not alias. */
tufrg_status tufrg_project(tufrg_ctx* ctx, const double* y_dev, double* v_dev,
                           void* cuda_stream);

/* Step ii with Fermi-surface-refined loop cells (Sec. 3: the paper
 * integrates each loop with an adaptive cubature; the refinement rule is a
 * reading).  The loop sums are the midpoint rule on the fine-grid cells;
 * below the scale lambda_on a cell p is refined for a transfer momentum l
 * when one of its propagators xi(k + l/2), xi(k - l/2), at the cell's centre
 * and four corners, changes sign or comes within kappa * Lambda of zero, and
 * its midpoint value is then replaced by the average over s x s sub-points
 * (s odd: they lie on the grid of s * nf points per direction).  Applies to
 * every later loop evaluation of the context (tufrg_loops, tufrg_rhs, flows,
 * row loops); s = 1, kappa = 0 or lambda_on = 0 switch it off.  Device tables
 * of (s nf)^2 (Nff + 1) numbers in the context's arithmetic type.
 * TUFRG_ERR_ARG for s even or outside 1..9, negative or non-finite kappa or
 * lambda_on, more than 512 parity-allowed pairs, or tables above 16 GiB. */
tufrg_status tufrg_set_refinement(tufrg_ctx* ctx, int32_t s, double kappa, double lambda_on,
                                  void* cuda_stream);

/* Step i from precomputed projection tensors (App. C; Sec. 2.5: the
 * scale-independent parts of the projections computed once and reused at
 * every scale).  Every cross projection is a linear map of the source
 * channel's propagator, B[Phi^B']_mn(l) = sum_{q,m',n'} A^{B,B'}_{mn,m'n'}(q, l)
 * B'_m'n'(q); three of the six tensors are stored, (P,C), (C,P), (D,C), the
 * others follow from the pair relations of App. C.  The tensors hold
 * 3 (Nl Nff^2)^2 numbers in the context's arithmetic type (FP64, or FP32 for
 * the mixed-precision contexts): bases of up to 9 form factors only.
 *
 * tufrg_atensor_bytes: device bytes the tensors take (host computation);
 *   TUFRG_ERR_ARG for more than 9 form factors.
 * tufrg_atensor_build: allocates (once) and computes the tensors from the
 *   projection terms, enqueued on cuda_stream; TUFRG_ERR_ARG if they would
 *   exceed 48 GiB, TUFRG_ERR_OOM if the device has no room.
 * tufrg_project_atensor: as tufrg_project (same layouts and result up to
 *   rounding), V = V0 + own + A y; TUFRG_ERR_STATE before
 *   tufrg_atensor_build.  The tensors are read once per call (HBM bound). */
tufrg_status tufrg_atensor_bytes(const tufrg_ctx* ctx, int64_t* bytes);
tufrg_status tufrg_atensor_build(tufrg_ctx* ctx, void* cuda_stream);
tufrg_status tufrg_project_atensor(tufrg_ctx* ctx, const double* y_dev, double* v_dev,
                                   void* cuda_stream);

/* Step iii, Eqs. (matmul-P/C/D), per l:
 *   dP = V^P chi^pp V^P, dC = -V^C chi^ph V^C,
 *   dD = 2 V^D chi^ph V^D - V^C chi^ph V^D - V^D chi^ph V^C.
 * v_dev: [3][Nl][Nff][Nff]; chi_dot_dev: [2][Nl][Nff][Nff];
 * dy_dev: [3][Nl][Nff][Nff] (may not alias the inputs). */
tufrg_status tufrg_products(tufrg_ctx* ctx, const double* v_dev, const double* chi_dot_dev,
                            double* dy_dev, void* cuda_stream);

/* Steps i-iii: dy/dLambda at scale lambda.  y_dev, dy_dev: [3][Nl][Nff][Nff];
 * may not alias.  Uses the context's workspace: calls on one context must be
 * stream-ordered (not concurrent).  The kernels run on the context's own
 * stream, ordered after the work on cuda_stream and before later work on it;
 * they are captured into a CUDA graph on the first call with a given
 * (y_dev, dy_dev) pair and replayed at the pair's later calls; the graphs of
 * the four most recently used pairs are kept (a caller double-buffering its
 * states replays both), a fifth pair replaces the least recently used one.
 * The first call with a pair is therefore slower and should not fall inside
 * a stream capture of the caller. */
tufrg_status tufrg_rhs(tufrg_ctx* ctx, double lambda, const double* y_dev, double* dy_dev,
                       void* cuda_stream);

/* Sec. 3/4: integrates the flow in s = ln Lambda from opts->lambda0 down to
 * opts->lambda_min, or until max |B| exceeds opts->threshold; the critical
 * scale is then located on the cubic Hermite dense output by bisection and
 * the state is returned there, with the classification of its largest
 * element.  y_dev: in = initial state (zeros: bare U), out = final state.
 * Equivalent to tufrg_flow_init + tufrg_flow_step(max_steps) +
 * tufrg_flow_state.  Running out of max_steps is not an error: the result
 * then has finished = 0 and the flow can be resumed (lambda0 = lambda_c,
 * h0 = h_next).  Blocks until done. */
tufrg_status tufrg_flow(tufrg_ctx* ctx, const tufrg_flow_opts* opts, double* y_dev,
                        tufrg_result* res, void* cuda_stream);

/* Stepwise flow (resume, external control, timing of single steps).  The
 * integrator state lives in the context (one flow per context at a time).
 * tufrg_flow_init copies y0_dev, takes the options (checkpoint scales are
 * copied; checkpoint_states_dev is kept) and evaluates the first stage
 * (one right-hand side).  Blocks until done. */
tufrg_status tufrg_flow_init(tufrg_ctx* ctx, const tufrg_flow_opts* opts, const double* y0_dev,
                             void* cuda_stream);

/* Performs up to n_steps step attempts (DoPri5: accepted or rejected, 6
 * right-hand sides each; RK4: n_steps steps of 4), stopping early when the
 * flow finishes; a threshold crossing is resolved (Lambda_c and the state
 * there) inside the step that crosses it.  res (may be NULL) receives the
 * progress (classification fields are not filled).  Blocks until done. */
tufrg_status tufrg_flow_step(tufrg_ctx* ctx, int32_t n_steps, tufrg_result* res,
                             void* cuda_stream);

/* Copies the integrator's current state (at Lambda_c after a divergence)
 * into y_dev ([3][Nl][Nff][Nff], may be NULL) and fills res including the
 * classification of the largest element.  Blocks until done. */
tufrg_status tufrg_flow_state(tufrg_ctx* ctx, double* y_dev, tufrg_result* res,
                              void* cuda_stream);

/* Allocation-free variant of tufrg_loops.  The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory -- code
 * whose device memory belongs to another allocator and may not call
 * cudaMalloc itself (a plugin hosted by another framework, a process held to
 * a budget reserved at start-up), or a latency-critical loop that must not
 * allocate once running.  It needs no context: from the parameters p (host)
 * it rebuilds the scale-independent tables and runs the FP64 loop
 * contraction (p->precision is ignored) entirely inside one static device
 * array of 16 MiB, which every GPU that loads the library holds until the
 * process exits.  The caller passes p, lambda > 0 and the output
 * chi_dot_dev [2][Nl][Nff][Nff] (device); results equal tufrg_loops up to
 * rounding.
 *  - Problems whose tables exceed the array (e.g. fine grids much beyond
 *    200 x 200 at Nff = 13) return TUFRG_ERR_ARG before any device work.
 *  - The first call on a device looks up the array's device address with
 *    that device current; make that first call before any stream capture.
 *  - All calls share the array: calls that overlap on the GPU (other
 *    streams, other host threads) race and corrupt each other's results, so
 *    serialise them.  Each call rewrites every part of the array it reads.
 *  - Calls no cudaMalloc, cudaFree or other allocating CUDA routine. */
tufrg_status tufrg_loops_noalloc(const tufrg_params* p, double lambda, double* chi_dot_dev,
                                 void* cuda_stream);

/* Chemical potential for filling n (particles per site, both spins):
 * bisection on n(mu) = (2/Nf) sum_k [eps0_k < mu] (ties count 1/2) over the
 * nf_x x nf_y grid.  Host computation. */
tufrg_status tufrg_mu_for_density(double t, double tp, double n, int32_t nf_x,
                                  int32_t nf_y, double* mu_out);

/* Diagnostic of the failure path (no counterpart in the paper): enqueues
 * one bounded device wait of wait_us microseconds (1..100000) on a barrier
 * that nothing completes.  It runs out, sets the context's error word the
 * way a stalled tensor-core pipeline would, and returns; the next
 * tufrg_check then reports TUFRG_ERR_TIMEOUT and clears it, and the context
 * stays usable.  TUFRG_ERR_ARG for a null context, one without a workspace
 * or wait_us out of range. */
tufrg_status tufrg_selftest_wait(tufrg_ctx* ctx, int32_t wait_us, void* cuda_stream);

/* Diagnostic of the library's own FP64 <-> FP32 conversions (no counterpart
 * in the paper; the FP32 projections read an FP32 copy of the state made by
 * them): x_dev [n] doubles -> y32_dev [n] floats rounded to nearest even,
 * then y32_dev -> back_dev [n] doubles (exact).  Device pointers, enqueued
 * on cuda_stream.  TUFRG_ERR_ARG for null pointers or n < 0. */
tufrg_status tufrg_selftest_convert(const double* x_dev, float* y32_dev, double* back_dev,
                                    int64_t n, void* cuda_stream);

/* Synchronises the stream and reports device-side failures of earlier
 * asynchronous calls on this context: TUFRG_ERR_TIMEOUT if a bounded wait
 * inside a kernel (tensor-core pipeline barriers) gave up; the flag is then
 * cleared.  tufrg_flow* calls check it themselves. */
tufrg_status tufrg_check(tufrg_ctx* ctx, void* cuda_stream);

/* ---------------------------------------------------------------------
 * The loop contraction of one point split over several GPUs (Sec. 3: the
 * paper distributes the bosonic momenta l over its MPI ranks).  The unit of
 * work is the loop row: one per class of transfer momenta l under the
 * point-group elements that map l into the zone without a fold (App. C),
 * whose loops follow from the row's by the point-group representation.  A
 * rank computes the rows [row_begin, row_end) of its context; the caller
 * gathers the row loops of all ranks (one collective per right-hand side)
 * and finishes the right-hand side on every rank with the replicated state.
 * Row loops are FP64 [2][nrow][npair] (pp, then ph; for each row the
 * parity-allowed pairs m <= n in the basis order, times -1/4 / +1/4 as in
 * chi_dot), row-major, caller-owned device memory.
 *
 * tufrg_row_info: the context's nrow and npair (host outputs).
 * tufrg_shard_rows: the context's loop contraction computes only the rows
 *   [row_begin, row_end), 0 <= row_begin < row_end <= nrow (the whole range
 *   undoes the split).  Tensor-core precisions only (TUFRG_ERR_ARG for an
 *   FP64 context).  While a context is split, tufrg_loops, tufrg_rhs and the
 *   flows return TUFRG_ERR_STATE.
 * tufrg_loop_rows: rows [row_begin, row_end) of the row loops at the scale
 *   lambda into rows_dev (the other rows untouched).  Stream-ordered.
 * tufrg_rhs_from_rows: the right-hand side (projections, products) of y at
 *   lambda with the loops given by complete row loops rows_dev.  y, dy as in
 *   tufrg_rhs. */
tufrg_status tufrg_row_info(const tufrg_ctx* ctx, int32_t* nrow, int32_t* npair);
tufrg_status tufrg_shard_rows(tufrg_ctx* ctx, int32_t row_begin, int32_t row_end,
                              void* cuda_stream);
tufrg_status tufrg_loop_rows(tufrg_ctx* ctx, double lambda, double* rows_dev, void* cuda_stream);
tufrg_status tufrg_rhs_from_rows(tufrg_ctx* ctx, double lambda, const double* rows_dev,
                                 const double* y_dev, double* dy_dev, void* cuda_stream);

/* ---------------------------------------------------------------------
 * Tile autotuning.  The tensor-core loop contraction cuts each point's loop
 * sum into work items of kbps K-blocks (64 fine-grid points per K-block for
 * BF16X3, 32 for 3XTF32) per tile of 128 l-rows; persistent CTAs, one per
 * SM, take the items from a queue.  Small items balance the SMs better,
 * large ones cost fewer partial sums and pipeline restarts; an item holds at
 * most 4096 loop points (FP32 accumulation chains).  The tuner times
 * one loop contraction per candidate (CUDA events, after a warm-up) and
 * keeps the fastest.  Results depend on kbps only through the FP32
 * accumulation order (differences at the level of the precision's rounding).
 */
typedef struct {
  int32_t n_candidates;   /* candidates timed (<= 16) */
  int32_t kbps[16];       /* K-blocks per work item of each candidate */
  double ms[16];          /* its loop-contraction time (median of the repeats) */
  int32_t chosen;         /* index of the candidate kept */
  int32_t kbps_default;   /* the setup's heuristic choice (also a candidate) */
} tufrg_tune_report;

/* Autotunes the context's tensor-core loop contraction at scale lambda
 * (TUFRG_ERR_ARG for an FP64 context).  rep may be NULL.  Blocks. */
tufrg_status tufrg_autotune(tufrg_ctx* ctx, double lambda, tufrg_tune_report* rep,
                            void* cuda_stream);

/* ---------------------------------------------------------------------
 * Batches: many phase-diagram points (own t, t', mu, U, grids and bond
 * shells) advanced together.  Each step of the right-hand side is one
 * launch over all points (the loop contraction one persistent launch whose
 * work items come from every point); a batched flow keeps step control per
 * point on the device and runs each DoPri5 attempt of all points as one
 * captured CUDA graph.
 *
 * Packed layouts: point i's state occupies elements
 * [state_offset_i, state_offset_i + 3 Nl_i Nff_i^2) of a packed state array
 * ([3][Nl_i][Nff_i][Nff_i] as for a context); its loops occupy
 * [loop_offset_i, loop_offset_i + 2 Nl_i Nff_i^2) of a packed loop array.
 */
typedef struct tufrg_batch tufrg_batch;

/* Sets up n_points points (params: host array [n_points]).  All points use
 * the same precision.  Points with equal grids and bond lists share their
 * scale-independent tables.  Blocks until the tables are on the device. */
tufrg_status tufrg_batch_setup(int32_t n_points, const tufrg_params* params, void* cuda_stream,
                               tufrg_batch** out);

void tufrg_batch_destroy(tufrg_batch* b);

/* Point sizes and packed offsets (any output may be NULL).  point = -1
 * gives the totals: *state_offset = packed state elements, *loop_offset =
 * packed loop elements, *nl = number of points. */
tufrg_status tufrg_batch_dims(const tufrg_batch* b, int32_t point, int32_t* nl, int32_t* nff,
                              int64_t* state_offset, int64_t* loop_offset);

/* Loops (Eq. chis) of every point, point i at scale lambda[i] (host array);
 * chi_dot_dev: packed loop array. */
tufrg_status tufrg_batch_loops(tufrg_batch* b, const double* lambda, double* chi_dot_dev,
                               void* cuda_stream);

/* Right-hand sides dy/dLambda of every point at its scale lambda[i];
 * y_dev, dy_dev: packed state arrays (may not alias). */
tufrg_status tufrg_batch_rhs(tufrg_batch* b, const double* lambda, const double* y_dev,
                             double* dy_dev, void* cuda_stream);

/* Flows of every point with the options of tufrg_flow (DoPri5 only; no
 * checkpoints; fp64_above must be 0).  Each point has its own step size,
 * acceptance and stop; a finished point does no further work.  The loop
 * runs until every point has finished or max_steps attempts were made.
 * y_dev: packed state, in = initial states, out = final states (at Lambda_c
 * for diverged points).  res: host array [n_points]; status: host array
 * [n_points] of each point's tufrg_status (may be NULL).  The return value
 * is the first failing point's status (TUFRG_ERR_TIMEOUT if a bounded wait
 * of the loop kernel gave up); a point that failed (non-finite state, step
 * underflow) stops there and the others go on.  Blocks. */
tufrg_status tufrg_batch_flow(tufrg_batch* b, const tufrg_flow_opts* opts, double* y_dev,
                              tufrg_result* res, int32_t* status, void* cuda_stream);

/* Autotunes the batch's persistent loop contraction (see tufrg_autotune),
 * every point at scale lambda. */
tufrg_status tufrg_batch_autotune(tufrg_batch* b, double lambda, tufrg_tune_report* rep,
                                  void* cuda_stream);

/* As tufrg_profile_loops, for the persistent contraction over all points. */
tufrg_status tufrg_batch_profile_loops(tufrg_batch* b, double lambda, int32_t n,
                                       double* kernel_ms, double* stage_ms, void* cuda_stream);

/* As tufrg_check, for the batch's kernels. */
tufrg_status tufrg_batch_check(tufrg_batch* b, void* cuda_stream);

/* ---------------------------------------------------------------------
 * Learned loop surrogate (not part of the paper's method).  A multilayer
 * perceptron predicts, per transfer momentum l of the coarse grid, the
 * targets
 *   Lambda (1 + Lambda) chi_dot_mn(l)
 * of the parity-allowed pairs m <= n of both loops (pp first, then ph, each
 * in the context's pair order; the other entries follow by symmetry or
 * vanish): n_out = 2 Npair outputs.  Its inputs (l_x, l_y, ln Lambda,
 * t', mu) enter scaled as
 *   x = (l_x/pi, l_y/pi, (ln Lambda - ln 0.1)/4.6, (t' + 0.225)/0.225,
 *        (mu + 0.9)/0.9),
 * then a fixed embedding maps x to 25 features (x; cos and sin of k pi x_0
 * and of k pi x_1 for k = 1..4, as the loops are periodic in l; x_2^2,
 * x_2^3, x_2 x_3, x_2 x_4), followed by `depth` hidden layers of `width`
 * SiLU units and a linear output layer whose outputs are standardised:
 * the network predicts (target - shift) / scale per output, shift and scale
 * being the mean and standard deviation of the first training set (identity
 * before that).  Forward and backward passes run on
 * tcgen05 tensor cores with BF16 hi/lo operand pairs (three products, as
 * the loop contraction) and FP32 accumulation; Adam keeps FP32 master
 * weights.  In a flow the surrogate replaces the loop contraction while an
 * exact-loop judge, run every judge_every accepted steps (and at the
 * start), finds its relative max-norm error at most tol; after the first
 * rejection the flow uses the exact loops to the end.
 *
 * Parameters are flattened layer by layer: W ([n_out][n_in] row-major),
 * then the bias.  x_dev: float [n][5]; t_dev, y_dev: float [n][n_out].
 */
typedef struct tufrg_surrogate tufrg_surrogate;

/* n_out <= 512, width a multiple of 64 (<= 512), 1 <= depth <= 8; weights
 * He-uniform from the seed, biases zero.  Blocks. */
tufrg_status tufrg_surrogate_create(int32_t n_out, int32_t width, int32_t depth, uint64_t seed,
                                    tufrg_surrogate** out);
void tufrg_surrogate_destroy(tufrg_surrogate* s);
tufrg_status tufrg_surrogate_n_params(const tufrg_surrogate* s, int64_t* n);
/* copy the FP32 master parameters to / from host memory.  Blocks. */
tufrg_status tufrg_surrogate_get_params(tufrg_surrogate* s, float* params, void* cuda_stream);
tufrg_status tufrg_surrogate_set_params(tufrg_surrogate* s, const float* params,
                                        void* cuda_stream);

/* The output standardisation (host arrays [n_out]).  set: shift and scale
 * both NULL restore the identity (the next training set then sets them);
 * scale > 0.  Block. */
tufrg_status tufrg_surrogate_get_scaling(tufrg_surrogate* s, float* shift, float* scale,
                                         void* cuda_stream);
tufrg_status tufrg_surrogate_set_scaling(tufrg_surrogate* s, const float* shift,
                                         const float* scale, void* cuda_stream);

/* Training samples of one scale: the exact loops of ctx at lambda (the
 * context's precision) as Nl rows of inputs x_dev [Nl][5] and targets
 * t_dev [Nl][n_out] (n_out must be 2 Npair of ctx). */
tufrg_status tufrg_surrogate_samples(tufrg_ctx* ctx, const tufrg_surrogate* s, double lambda,
                                     float* x_dev, float* t_dev, void* cuda_stream);

/* Predicted targets y_dev [n][n_out] (standardisation undone) for inputs
 * x_dev [n][5]. */
tufrg_status tufrg_surrogate_predict(tufrg_surrogate* s, const float* x_dev, int64_t n,
                                     float* y_dev, void* cuda_stream);

/* Mean squared error of the standardised outputs against the standardised
 * targets over n samples (n <= 65536) and its gradient with respect to the
 * flattened parameters (host arrays; grad may be NULL).  Blocks. */
tufrg_status tufrg_surrogate_loss_grad(tufrg_surrogate* s, const float* x_dev,
                                       const float* t_dev, int64_t n, double* loss,
                                       float* grad, void* cuda_stream);

/* Adam (beta 0.9, 0.999, eps 1e-8) on mini-batches of `batch` samples
 * drawn without replacement (seeded shuffle per epoch), learning rate lr
 * with cosine decay to lr/100.  loss_hist (host, may be NULL) receives the
 * mean mini-batch loss of each epoch.  Blocks. */
tufrg_status tufrg_surrogate_train(tufrg_surrogate* s, const float* x_dev, const float* t_dev,
                                   int64_t n, int32_t epochs, int32_t batch, double lr,
                                   uint64_t seed, double* loss_hist, void* cuda_stream);

/* Lets the DoPri5 flows of ctx use the surrogate for the loops (s = NULL
 * detaches).  judge_every >= 1 accepted steps between exact judgements;
 * tol > 0 the largest accepted relative max-norm error of the loops.  The
 * surrogate's work buffers serve one flow at a time. */
tufrg_status tufrg_surrogate_attach(tufrg_ctx* ctx, tufrg_surrogate* s, int32_t judge_every,
                                    double tol);

/* Measurement: runs n loop contractions of the context at scale lambda (up
 * to the loops of the rows, as a right-hand side does) and returns the mean
 * duration of the contraction kernel itself (kernel_ms; CUDA events recorded
 * around its launch on its stream) and of the whole loop stage -- per-scale
 * table, contraction, split-K combination -- (stage_ms).  Blocks. */
tufrg_status tufrg_profile_loops(tufrg_ctx* ctx, double lambda, int32_t n, double* kernel_ms,
                                 double* stage_ms, void* cuda_stream);

const char* tufrg_status_string(tufrg_status s);

/* The CUDA error behind the calling thread's last TUFRG_ERR_CUDA or
 * TUFRG_ERR_OOM: its name and the library source location of the failing
 * call ("" if none). */
const char* tufrg_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TUFRG_H */
