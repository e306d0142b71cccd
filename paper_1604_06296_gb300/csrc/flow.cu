// Sec. 3/4: integration of the flow dy/ds = Lambda dy/dLambda, s = ln Lambda,
// from ln Lambda0 downwards with Dormand-Prince 5(4) (published tableau,
// Dormand & Prince 1980) or fixed-step RK4, until max |B| exceeds the
// threshold or Lambda_min is reached.  The critical scale is the first point
// where max |B| reaches the threshold on the cubic Hermite interpolant of the
// crossing step, located by 100 bisection steps; the state there is
// classified by the channel / l / (m, n) of its largest element.
//
// Step control runs on the device (one thread), so one DoPri5 attempt is a
// fixed sequence of kernels -- six stages of (combination, right-hand side),
// error norm, control, accept -- captured once as a CUDA graph on the
// library's own stream and replayed; the host reads a small status block
// after each attempt.  Control:
//   err = max_i |h sum_j e_j k_j| / (atol + rtol max(|y_i|, |y_new,i|))
//   accept if err <= 1; factor 0.9 err^(-1/5) clipped to [0.2, 5], no growth
//   right after a rejection; the next step is clipped to land on ln Lambda_min.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "device_util.cuh"
#include "flow_common.cuh"

namespace tufrg {
namespace {

// Element-wise kernels: 256 threads, up to kPer elements per thread with all
// their loads in flight -- as many as keep ~8 CTAs per SM busy, so a small
// state still spreads over every SM.
constexpr int kPer = 8;

__host__ __device__ inline int per_thread(size_t n) {
  const size_t p = n / (256 * 152 * 8);
  return p < 1 ? 1 : (p > kPer ? kPer : (int)p);
}

// out = y + h * sum_j a_j k_j (and, when out32 is given, its FP32 copy for
// the FP32 projections); one thread also publishes Lambda for the RHS
__global__ void combo_kernel(const double* __restrict__ y, double* __restrict__ out, Combo cb,
                             const FlowCtl* __restrict__ ctl, double* __restrict__ lam,
                             size_t n, int set_lambda, float* __restrict__ out32 = nullptr) {
  const double h = ctl->h;
  if (set_lambda && blockIdx.x == 0 && threadIdx.x == 0) {
    const double L = exp(ctl->s + cb.c * h);
    lam[0] = L;
    lam[1] = L;
  }
  const int per = per_thread(n);
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const size_t i = ((size_t)blockIdx.x * per + u) * blockDim.x + threadIdx.x;
    if (u >= per || i >= n) break;
    const double acc = combo_sum(cb, i);
    const double v = y[i] + h * acc;
    out[i] = v;
    if (out32) out32[i] = d2f(v);
  }
}

// the scale of a stage: Lambda = exp(s + c h), for the loops and for dy/ds
__global__ void stage_lambda_kernel(const FlowCtl* __restrict__ ctl, double cnode,
                                    double* __restrict__ lam) {
  const double L = exp(ctl->s + cnode * ctl->h);
  lam[0] = L;
  lam[1] = L;
}

__global__ void error_kernel(const double* __restrict__ y, const double* __restrict__ ynew,
                             Combo e, FlowCtl* __restrict__ ctl, size_t n) {
  const double h = ctl->h, rtol = ctl->rtol, atol = ctl->atol;
  unsigned long long emax = 0, ymax = 0;
  int bad = 0;
  const int per = per_thread(n);
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const size_t i = ((size_t)blockIdx.x * per + u) * blockDim.x + threadIdx.x;
    if (u >= per || i >= n) break;
    const double acc = combo_sum(e, i);
    const double yn = ynew[i];
    const double sc = atol + rtol * fmax(fabs(y[i]), fabs(yn));
    // the ratio in FP32 (the step control needs a few digits of it; GB300's
    // FP64 division costs more than the rest of the kernel)
    const double r = (double)__fdiv_rn((float)fabs(h * acc), (float)sc);
    if (!isfinite(yn) || !isfinite(r)) bad = 1;
    emax = max(emax, abs_bits(r));
    ymax = max(ymax, abs_bits(yn));
  }
  if (bad) ctl->nonfinite = 1;
  block_max_u(emax, &ctl->err_u);
  block_max_u(ymax, &ctl->max_u);
}

__global__ void control_kernel(FlowCtl* c) { control_update(c); }

// on acceptance: keep the previous point for dense output and move on (FSAL)
__global__ void accept_kernel(double* __restrict__ y, const double* __restrict__ ynew,
                              double* __restrict__ yprev, double* __restrict__ k1,
                              const double* __restrict__ k7, double* __restrict__ k1prev,
                              const FlowCtl* __restrict__ ctl, size_t n) {
  if (!ctl->accepted) return;
  const int per = per_thread(n);
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const size_t i = ((size_t)blockIdx.x * per + u) * blockDim.x + threadIdx.x;
    if (u >= per || i >= n) break;
    yprev[i] = y[i];
    y[i] = ynew[i];
    k1prev[i] = k1[i];
    k1[i] = k7[i];
  }
}

// Interpolant of the last accepted step at s_fixed (or at the bisection
// midpoint when use_mid); writes it to out if non-null and, when track,
// accumulates max |value| into ctl->bis_u.
__global__ void hermite_kernel(const double* __restrict__ y0, const double* __restrict__ f0,
                               const double* __restrict__ y1, const double* __restrict__ f1,
                               FlowCtl* __restrict__ ctl, double s_fixed, int use_mid,
                               double* __restrict__ out, size_t n, int track) {
  const double s0 = ctl->s_prev, s1 = ctl->s;
  const double s = use_mid ? 0.5 * (ctl->bis_a + ctl->bis_b) : s_fixed;
  unsigned long long m = 0;
  const int per = per_thread(n);
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const size_t i = ((size_t)blockIdx.x * per + u) * blockDim.x + threadIdx.x;
    if (u >= per || i >= n) break;
    const double v = hermite(s0, y0[i], f0[i], s1, y1[i], f1[i], s);
    if (out) out[i] = v;
    m = max(m, abs_bits(v));
  }
  if (track) block_max_u(m, &ctl->bis_u);
}

__global__ void bisect_update_kernel(FlowCtl* c) {
  const double m = 0.5 * (c->bis_a + c->bis_b);
  const double g = __longlong_as_double((long long)c->bis_u);
  if (g > c->thr)
    c->bis_b = m;
  else
    c->bis_a = m;
  c->bis_u = 0;
}

__global__ void max_kernel(const double* __restrict__ y, FlowCtl* __restrict__ ctl, size_t n,
                           int check_finite) {
  unsigned long long m = 0;
  int bad = 0;
  const int per = per_thread(n);
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const size_t i = ((size_t)blockIdx.x * per + u) * blockDim.x + threadIdx.x;
    if (u >= per || i >= n) break;
    m = max(m, abs_bits(y[i]));
    if (check_finite && !isfinite(y[i])) bad = 1;
  }
  if (bad) ctl->nonfinite = 1;
  block_max_u(m, &ctl->max_u);
}

__global__ void argmax_kernel(const double* __restrict__ y, FlowCtl* __restrict__ ctl, size_t n) {
  const unsigned long long target = ctl->max_u;
  const int per = per_thread(n);
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const size_t i = ((size_t)blockIdx.x * per + u) * blockDim.x + threadIdx.x;
    if (u >= per || i >= n) break;
    if (abs_bits(y[i]) == target) atomicMin(&ctl->arg_u, (unsigned long long)i);
  }
}

double bits_to_double(unsigned long long u) {
  double d;
  std::memcpy(&d, &u, sizeof d);
  return d;
}

// CTAs of the element-wise kernels for n elements
int grid_for(size_t n) {
  const size_t per = (size_t)256 * per_thread(n);
  return (int)((n + per - 1) / per);
}

}  // namespace

// Integrator state kept in the context between tufrg_flow_* calls.
struct FlowState {
  bool initialized = false, finished = false, crossed = false;
  int method = TUFRG_DOPRI5;
  double threshold = 0.0;
  std::vector<std::pair<double, int>> cks;  // (ln Lambda, output slot), largest first
  size_t next_ck = 0;
  double* ck_out = nullptr;
  long long rk4_rhs = 0;
  FlowCtl* hc = nullptr;  // pinned host mirror of the control block
  double* base = nullptr;
  size_t bytes = 0;
  double *y, *k[7], *ytmp, *ynew, *yprev, *k1prev;
  FlowCtl* ctl = nullptr;
  cudaGraphExec_t attempt[3] = {nullptr, nullptr, nullptr};  // loops: context, FP64, surrogate
  double fp64_above = 0.0;
  double lambda_switch = 0.0;
  // the flow's state is point-group covariant (checked at the start; exact
  // loops keep it so): projections and products at the rows' representative
  // l only.  graphs_wedge: the setting the attempt graphs were captured with
  bool wedge = false, graphs_wedge = false;
  unsigned long long* cov = nullptr;  // [2]: covariance deviation and max |y| (device)
  // elements of the flow's vectors: the wedge layout [3][nrow][nff][nff]
  // (the state at the rows' representatives), or the full state
  size_t nflow = 0;
  // loop surrogate: accepted steps since the last judgement, the scale at
  // which the judge rejected it, right-hand sides it served, judgements
  int since_judge = 0;
  double lambda_sur_off = 0.0;
  long long n_rhs_sur = 0, n_judges = 0;
};

namespace {

tufrg_status ensure_buffers(tufrg_ctx* c) {
  if (!c->flow) {
    c->flow = new (std::nothrow) FlowState();
    if (!c->flow) return TUFRG_ERR_OOM;
  }
  FlowState& f = *c->flow;
  if (!f.hc) TUFRG_CUDA(cudaMallocHost((void**)&f.hc, sizeof(FlowCtl)));
  const size_t n = c->state_elems();
  const size_t need = sizeof(double) * n * 12 + 1024;
  if (f.bytes < need) {
    for (auto& g : f.attempt) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
    if (f.base) cudaFree(f.base);
    f.base = nullptr;
    f.bytes = 0;
    if (cudaMalloc((void**)&f.base, need) != cudaSuccess) return TUFRG_ERR_OOM;
    f.bytes = need;
  }
  double* p = f.base;
  f.y = p;
  for (int i = 0; i < 7; ++i) f.k[i] = p + n * (1 + i);
  f.ytmp = p + n * 8;
  f.ynew = p + n * 9;
  f.yprev = p + n * 10;
  f.k1prev = p + n * 11;
  f.ctl = (FlowCtl*)(p + n * 12);
  f.cov = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(f.ctl) + 512);
  static_assert(sizeof(FlowCtl) <= 512, "the covariance words follow the control block");
  return TUFRG_OK;
}

tufrg_status stage(tufrg_ctx* c, const double* y, double* out,
                   const std::vector<std::pair<double, const double*>>& terms, double cnode,
                   double* k_out, cudaStream_t st) {
  FlowState& f = *c->flow;
  Combo cb{};
  cb.nk = (int)terms.size();
  for (int j = 0; j < cb.nk; ++j) {
    cb.a[j] = terms[j].first;
    cb.k[j] = terms[j].second;
  }
  cb.c = cnode;
  const size_t n = f.nflow;
  // the stage's state on the projection stream (its consumer), its scale on
  // the loop stream: the loops start without waiting for the combination
  TUFRG_CUDA(cudaEventRecord(c->ev_stage, st));
  TUFRG_CUDA(cudaStreamWaitEvent(c->pstream, c->ev_stage, 0));
  // the FP32 projections' copy of the stage state, written by the combination
  float* y32 = rhs_arith(c, c->loop_prec) == TUFRG_FP64 ? nullptr : c->d_y32;
  combo_kernel<<<grid_for(n), 256, 0, c->pstream>>>(y, out, cb, f.ctl, c->d_lambda, n, 0, y32);
  stage_lambda_kernel<<<1, 1, 0, st>>>(f.ctl, cnode, c->d_lambda);
  TUFRG_CUDA(cudaGetLastError());
  return rhs_device(c, c->loop_prec, out, k_out, true, st, f.wedge, y32);
}

// One DoPri5 attempt: stages 2..7, error norm, control, accept.
tufrg_status enqueue_attempt(tufrg_ctx* c, cudaStream_t st) {
  FlowState& f = *c->flow;
  const size_t n = f.nflow;
  for (int i = 1; i < 7; ++i) {
    std::vector<std::pair<double, const double*>> t;
    for (int j = 0; j < i; ++j)
      if (kA[i][j] != 0.0) t.push_back({kA[i][j], f.k[j]});
    TUFRG_CHECK(stage(c, f.y, i == 6 ? f.ynew : f.ytmp, t, kC[i], f.k[i], st));
  }
  Combo ce{};
  for (int j = 0; j < 7; ++j)
    if (kB[j] != kBs[j]) {
      ce.a[ce.nk] = kB[j] - kBs[j];
      ce.k[ce.nk] = f.k[j];
      ++ce.nk;
    }
  const int G = grid_for(n);
  error_kernel<<<G, 256, 0, st>>>(f.y, f.ynew, ce, f.ctl, n);
  control_kernel<<<1, 1, 0, st>>>(f.ctl);
  accept_kernel<<<G, 256, 0, st>>>(f.y, f.ynew, f.yprev, f.k[0], f.k[6], f.k1prev, f.ctl, n);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status read_ctl(tufrg_ctx* c, cudaStream_t st) {
  FlowState& f = *c->flow;
  TUFRG_CUDA(cudaMemcpyAsync(f.hc, f.ctl, sizeof(FlowCtl), cudaMemcpyDeviceToHost, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

tufrg_status write_ctl(tufrg_ctx* c, const FlowCtl& v, cudaStream_t st) {
  FlowState& f = *c->flow;
  *f.hc = v;
  TUFRG_CUDA(cudaMemcpyAsync(f.ctl, f.hc, sizeof(FlowCtl), cudaMemcpyHostToDevice, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

// max |B| crossed the threshold inside [s, s_prev]: bisection on the Hermite
// interpolant, then the state at the crossing replaces y.
tufrg_status resolve_crossing(tufrg_ctx* c, cudaStream_t st) {
  FlowState& f = *c->flow;
  const size_t n = f.nflow;
  const int G = grid_for(n);
  FlowCtl cur = *f.hc;
  cur.bis_a = cur.s_prev;
  cur.bis_b = cur.s;
  cur.bis_u = 0;
  TUFRG_CHECK(write_ctl(c, cur, st));
  for (int it = 0; it < kBisect; ++it) {
    hermite_kernel<<<G, 256, 0, st>>>(f.yprev, f.k1prev, f.y, f.k[0], f.ctl, 0.0, 1, nullptr, n,
                                      1);
    bisect_update_kernel<<<1, 1, 0, st>>>(f.ctl);
  }
  TUFRG_CUDA(cudaGetLastError());
  TUFRG_CHECK(read_ctl(c, st));
  const double sc = f.hc->bis_b;
  hermite_kernel<<<G, 256, 0, st>>>(f.yprev, f.k1prev, f.y, f.k[0], f.ctl, sc, 0, f.ytmp, n, 0);
  TUFRG_CUDA(cudaGetLastError());
  TUFRG_CUDA(cudaMemcpyAsync(f.y, f.ytmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  FlowCtl fin = *f.hc;
  fin.s = sc;
  return write_ctl(c, fin, st);
}

tufrg_status checkpoints_in_last_step(tufrg_ctx* c, cudaStream_t st) {
  FlowState& f = *c->flow;
  const size_t n = f.nflow;
  while (f.next_ck < f.cks.size() && f.cks[f.next_ck].first >= f.hc->s &&
         f.cks[f.next_ck].first <= f.hc->s_prev) {
    // the full state of the checkpoint (a wedge-layout interpolant expanded)
    double* dst = f.ck_out + c->state_elems() * f.cks[f.next_ck].second;
    hermite_kernel<<<grid_for(n), 256, 0, st>>>(f.yprev, f.k1prev, f.y, f.k[0], f.ctl,
                                                f.cks[f.next_ck].first, 0,
                                                f.wedge ? f.ytmp : dst, n, 0);
    TUFRG_CUDA(cudaGetLastError());
    if (f.wedge) TUFRG_CHECK(launch_wedge_expand(c->view, f.ytmp, dst, st));
    ++f.next_ck;
  }
  return TUFRG_OK;
}

// The attempt graph of the current loop precision (captured on first use).
tufrg_status attempt_graph(tufrg_ctx* c, cudaStream_t st, cudaGraphExec_t* out) {
  FlowState& f = *c->flow;
  const int which = c->loop_prec == TUFRG_FP64 ? 1 : (c->loop_prec == kLoopSurrogate ? 2 : 0);
  if (!f.attempt[which]) {
    cudaGraph_t g = nullptr;
    TUFRG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    tufrg_status s = enqueue_attempt(c, st);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s != TUFRG_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    TUFRG_CUDA(e);
    e = cudaGraphInstantiate(&f.attempt[which], g, 0);
    cudaGraphDestroy(g);
    TUFRG_CUDA(e);
  }
  *out = f.attempt[which];
  return TUFRG_OK;
}

// Exact-loop judgement of the surrogate at the current scale; on rejection
// the flow continues with the exact loops and k1 is recomputed with them.
tufrg_status judge(tufrg_ctx* c, double s, bool at_start, cudaStream_t st) {
  FlowState& f = *c->flow;
  TUFRG_CHECK(launch_set_scalar(c->d_lambda, std::exp(s), st));
  double rel = 0.0;
  TUFRG_CHECK(surrogate_judge(c->sur, c, c->p.precision, &rel, st));
  ++f.n_judges;
  f.since_judge = 0;
  if (rel <= c->sur_tol) {
    c->loop_prec = kLoopSurrogate;
    return TUFRG_OK;
  }
  c->loop_prec = c->p.precision;
  f.lambda_sur_off = std::exp(s);
  if (!at_start) {  // FSAL stage of the current point with the exact loops
    TUFRG_CHECK(stage(c, f.y, f.ytmp, {}, 0.0, f.k[0], st));
    TUFRG_CUDA(cudaStreamSynchronize(st));
  }
  return TUFRG_OK;
}

tufrg_status dopri5_steps(tufrg_ctx* c, int n_steps, cudaStream_t st) {
  FlowState& f = *c->flow;
  for (int i = 0; i < n_steps && !f.finished; ++i) {
    if (c->loop_prec == kLoopSurrogate && f.since_judge >= c->sur_every)
      TUFRG_CHECK(judge(c, f.hc->s, false, st));
    const bool sur = c->loop_prec == kLoopSurrogate;
    cudaGraphExec_t g = nullptr;
    TUFRG_CHECK(attempt_graph(c, st, &g));
    TUFRG_CUDA(cudaGraphLaunch(g, st));
    TUFRG_CHECK(read_ctl(c, st));
    if (sur) {
      f.n_rhs_sur += 6;
      if (f.hc->accepted) ++f.since_judge;
    }
    if (f.hc->accepted && f.fp64_above > 0.0 && c->loop_prec != TUFRG_FP64 &&
        f.hc->ymax_last > f.fp64_above) {
      c->loop_prec = TUFRG_FP64;  // near the divergence: the remaining loops in FP64
      f.lambda_switch = std::exp(f.hc->s);
    }
    if (f.hc->status != TUFRG_OK) {
      f.finished = true;
      return (tufrg_status)f.hc->status;
    }
    if (f.hc->accepted) TUFRG_CHECK(checkpoints_in_last_step(c, st));
    if (f.hc->crossed) {
      f.crossed = true;
      f.finished = true;
      TUFRG_CHECK(resolve_crossing(c, st));
    } else if (f.hc->done) {
      f.finished = true;
    }
  }
  return TUFRG_OK;
}

// Classic RK4 with equal steps; stops early when max |y| exceeds the threshold.
tufrg_status rk4_steps(tufrg_ctx* c, int n_steps, cudaStream_t st) {
  FlowState& f = *c->flow;
  const size_t n = f.nflow;
  const int G = grid_for(n);
  for (int i = 0; i < n_steps && !f.finished; ++i) {
    if ((f.hc->s_end - f.hc->s) * f.hc->dir <= 1e-12) {  // reached ln Lambda_min
      f.finished = true;
      break;
    }
    TUFRG_CHECK(stage(c, f.y, f.ytmp, {}, 0.0, f.k[0], st));
    TUFRG_CHECK(stage(c, f.y, f.ytmp, {{0.5, f.k[0]}}, 0.5, f.k[1], st));
    TUFRG_CHECK(stage(c, f.y, f.ytmp, {{0.5, f.k[1]}}, 0.5, f.k[2], st));
    TUFRG_CHECK(stage(c, f.y, f.ytmp, {{1.0, f.k[2]}}, 1.0, f.k[3], st));
    f.rk4_rhs += 4;
    Combo cb{};
    cb.nk = 4;
    const double w[4] = {1.0 / 6, 2.0 / 6, 2.0 / 6, 1.0 / 6};
    for (int j = 0; j < 4; ++j) {
      cb.a[j] = w[j];
      cb.k[j] = f.k[j];
    }
    combo_kernel<<<G, 256, 0, st>>>(f.y, f.ynew, cb, f.ctl, c->d_lambda, n, 0);
    TUFRG_CUDA(cudaGetLastError());
    TUFRG_CUDA(cudaMemcpyAsync(f.y, f.ynew, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    TUFRG_CHECK(read_ctl(c, st));
    FlowCtl adv = *f.hc;
    adv.s_prev = adv.s;
    adv.s = adv.s + adv.h;
    adv.n_acc += 1;
    adv.max_u = 0;
    adv.nonfinite = 0;
    TUFRG_CHECK(write_ctl(c, adv, st));
    max_kernel<<<G, 256, 0, st>>>(f.y, f.ctl, n, 1);
    TUFRG_CUDA(cudaGetLastError());
    TUFRG_CHECK(read_ctl(c, st));
    if (f.hc->nonfinite) {
      f.finished = true;
      return TUFRG_ERR_NONFINITE;
    }
    if (bits_to_double(f.hc->max_u) > f.threshold) {
      f.crossed = true;
      f.finished = true;
    }
  }
  return TUFRG_OK;
}

void fill_progress(tufrg_ctx* c, tufrg_result* r) {
  FlowState& f = *c->flow;
  r->lambda_c = std::exp(f.hc->s);
  r->h_next = std::fabs(f.hc->h);
  r->diverged = f.crossed ? 1 : 0;
  r->finished = f.finished ? 1 : 0;
  r->n_accepted = f.hc->n_acc;
  r->n_rejected = f.hc->n_rej;
  r->n_rhs = f.method == TUFRG_RK4 ? f.rk4_rhs : 1 + f.hc->n_rhs;
  r->lambda_switch = f.lambda_switch;
  r->lambda_surrogate_off = f.lambda_sur_off;
  r->n_rhs_surrogate = f.n_rhs_sur;
  r->n_judges = f.n_judges;
}

}  // namespace

void flow_drop_graphs(tufrg_ctx* c) {
  for (auto& r : c->rhs_graphs) {
    if (r.exec) cudaGraphExecDestroy(r.exec);
    r = tufrg_ctx::RhsGraph{};
  }
  if (!c->flow) return;
  for (auto& g : c->flow->attempt) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

void free_flow(tufrg_ctx* c) {
  if (!c->flow) return;
  FlowState& f = *c->flow;
  for (auto& g : f.attempt)
    if (g) cudaGraphExecDestroy(g);
  if (f.base) cudaFree(f.base);
  if (f.hc) cudaFreeHost(f.hc);
  delete c->flow;
  c->flow = nullptr;
}

tufrg_status flow_init(tufrg_ctx* c, const tufrg_flow_opts* o, const double* y0,
                       cudaStream_t st) {
  TUFRG_CHECK(ensure_buffers(c));
  FlowState& f = *c->flow;
  f.initialized = false;
  f.finished = f.crossed = false;
  f.method = o->method;
  f.threshold = o->threshold;
  f.fp64_above = o->fp64_above;
  f.lambda_switch = 0.0;
  f.since_judge = 0;
  f.lambda_sur_off = 0.0;
  f.n_rhs_sur = f.n_judges = 0;
  c->loop_prec = c->p.precision;  // every flow starts in the context's precision
  f.rk4_rhs = 0;
  f.cks.clear();
  for (int i = 0; i < o->n_checkpoints; ++i) f.cks.push_back({std::log(o->checkpoints[i]), i});
  std::sort(f.cks.begin(), f.cks.end(), [](auto& a, auto& b) { return a.first > b.first; });
  f.next_ck = 0;
  f.ck_out = o->checkpoint_states_dev;
  const size_t n = c->state_elems();

  FlowCtl h0{};
  h0.s = std::log(o->lambda0);
  h0.s_end = std::log(o->lambda_min);
  h0.dir = -1.0;
  h0.rtol = o->rtol;
  h0.atol = o->atol;
  h0.thr = o->threshold;
  h0.h = -std::fabs(o->h0);
  if (o->method == TUFRG_RK4) {
    const int steps = std::max(1, (int)std::lround((h0.s - h0.s_end) / std::fabs(o->h0)));
    h0.h = (h0.s_end - h0.s) / steps;
  } else if (h0.s + h0.h < h0.s_end) {
    h0.h = h0.s_end - h0.s;
  }
  TUFRG_CUDA(cudaMemcpyAsync(f.y, y0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  // the wedge when the initial state is covariant (the bare start, zeros, is)
  // and every loop is exact (a surrogate's loops are not covariant): the
  // flow then integrates the state at the rows' representatives only
  f.wedge = false;
  if (!c->sur) {
    TUFRG_CHECK(launch_covariance_check(c->view, f.y, f.cov, st));
    unsigned long long h[2] = {0, 0};
    TUFRG_CUDA(cudaMemcpyAsync(h, f.cov, sizeof(h), cudaMemcpyDeviceToHost, st));
    TUFRG_CUDA(cudaStreamSynchronize(st));
    double dev, amax;
    std::memcpy(&dev, &h[0], 8);
    std::memcpy(&amax, &h[1], 8);
    f.wedge = dev <= 1e-13 * amax;
  }
  f.nflow = n;
  if (f.wedge) {
    TUFRG_CHECK(launch_wedge_compress(c->view, f.y, f.ynew, st));
    f.nflow = c->view.wstate_elems;
    TUFRG_CUDA(cudaMemcpyAsync(f.y, f.ynew, sizeof(double) * f.nflow, cudaMemcpyDeviceToDevice,
                               st));
  }
  if (f.wedge != f.graphs_wedge) {
    for (auto& g : f.attempt) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
    f.graphs_wedge = f.wedge;
  }
  TUFRG_CHECK(write_ctl(c, h0, st));
  if (o->method == TUFRG_DOPRI5) {
    if (c->sur) {  // the surrogate's buffers may have moved: capture afresh
      flow_drop_graphs(c);
      TUFRG_CHECK(judge(c, h0.s, true, st));
      if (c->loop_prec == kLoopSurrogate) f.n_rhs_sur = 1;  // the first stage below
    }
    TUFRG_CHECK(stage(c, f.y, f.ytmp, {}, 0.0, f.k[0], st));  // k1 = f(s0, y0)
    TUFRG_CUDA(cudaStreamSynchronize(st));
  }
  f.initialized = true;
  return TUFRG_OK;
}

tufrg_status flow_step(tufrg_ctx* c, int n_steps, tufrg_result* r, cudaStream_t st) {
  if (!c->flow || !c->flow->initialized) return TUFRG_ERR_STATE;
  FlowState& f = *c->flow;
  tufrg_status s = f.method == TUFRG_RK4 ? rk4_steps(c, n_steps, st) : dopri5_steps(c, n_steps, st);
  if (r) {
    TUFRG_CHECK(read_ctl(c, st));
    fill_progress(c, r);
  }
  return s;
}

tufrg_status flow_state(tufrg_ctx* c, double* y_out, tufrg_result* r, cudaStream_t st) {
  if (!c->flow || !c->flow->initialized) return TUFRG_ERR_STATE;
  FlowState& f = *c->flow;
  const size_t n = c->state_elems();
  const int G = grid_for(n);
  TUFRG_CHECK(read_ctl(c, st));
  FlowCtl cur = *f.hc;
  cur.max_u = 0;
  cur.arg_u = ~0ull;
  TUFRG_CHECK(write_ctl(c, cur, st));
  // the full state (a wedge-layout state expanded to every l)
  const double* yfull = f.y;
  if (f.wedge) {
    TUFRG_CHECK(launch_wedge_expand(c->view, f.y, f.ytmp, st));
    yfull = f.ytmp;
  }
  max_kernel<<<G, 256, 0, st>>>(yfull, f.ctl, n, 0);
  argmax_kernel<<<G, 256, 0, st>>>(yfull, f.ctl, n);
  TUFRG_CUDA(cudaGetLastError());
  if (y_out)
    TUFRG_CUDA(cudaMemcpyAsync(y_out, yfull, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  TUFRG_CHECK(read_ctl(c, st));
  if (r) {
    fill_progress(c, r);
    const size_t per_ch = (size_t)c->nl * c->nff * c->nff;
    const unsigned long long idx = f.hc->arg_u;
    r->max_abs = bits_to_double(f.hc->max_u);
    if (idx < n) {
      r->channel = (int32_t)(idx / per_ch);
      size_t rem = idx % per_ch;
      r->l_index = (int32_t)(rem / ((size_t)c->nff * c->nff));
      rem %= (size_t)c->nff * c->nff;
      r->m = (int32_t)(rem / c->nff);
      r->n = (int32_t)(rem % c->nff);
    } else {
      r->channel = r->l_index = r->m = r->n = -1;
    }
  }
  return TUFRG_OK;
}

}  // namespace tufrg
