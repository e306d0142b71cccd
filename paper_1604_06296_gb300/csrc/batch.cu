// Batches of phase-diagram points (tufrg_batch_*) and the tile autotuner.
//
// Each step of the right-hand side runs once for all points of the batch:
// the tensor-core loop contraction is one persistent launch whose work items
// come from every point, the table, reduction, projection and product
// kernels are multi-point launches (CTAs of a point found from a prefix
// table).  A batched flow integrates every point with DoPri5 in s = ln Lambda
// (the control law of the single-point flow, one control block per point):
// one attempt of all points -- six stages of (combination, right-hand side),
// error norms, control, accept -- is one captured CUDA graph; points that
// have finished are skipped by every kernel (their work items return at
// once), so the graph stays fixed while the work shrinks.  Threshold
// crossings are resolved after the loop by a bisection on each crossed
// point's Hermite interpolant (its last step is kept intact once it stops).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "device_util.cuh"
#include "flow_common.cuh"

namespace tufrg {
namespace {

constexpr int kChunk = 2048;  // state elements per CTA of the element-wise flow kernels
constexpr int kFlowThreads = 256;

struct Seg {
  long long off, len;  // the point's elements in the packed state
};

// out = y + h sum_j a_j k_j and its FP32 copy out32 (the FP32 projections'
// input) for every active point
__global__ void bcombo_kernel(const double* __restrict__ y, double* __restrict__ out, Combo cb,
                              const FlowCtl* __restrict__ ctl, double* __restrict__ lam,
                              const Seg* __restrict__ seg, const int* __restrict__ prefix, int n,
                              int set_lambda, float* __restrict__ out32) {
  const int p = point_of(prefix, n, blockIdx.x);
  const FlowCtl& c = ctl[p];
  if (c.done) return;
  const double h = c.h;
  const int chunk = blockIdx.x - prefix[p];
  if (set_lambda && chunk == 0 && threadIdx.x == 0) {
    const double L = exp(c.s + cb.c * h);
    lam[2 * p] = L;
    lam[2 * p + 1] = L;
  }
  const long long b = seg[p].off + (long long)chunk * kChunk;
  const long long e = min(b + kChunk, seg[p].off + seg[p].len);
#pragma unroll
  for (int u = 0; u < kChunk / kFlowThreads; ++u) {
    const long long i = b + u * kFlowThreads + threadIdx.x;
    if (i >= e) break;
    const double acc = combo_sum(cb, i);
    const double v = y[i] + h * acc;
    out[i] = v;
    out32[i] = d2f(v);
  }
}

// the scales of a stage of every active point
__global__ void bstage_lambda_kernel(const FlowCtl* __restrict__ ctl, double cnode,
                                     double* __restrict__ lam, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || ctl[p].done) return;
  const double L = exp(ctl[p].s + cnode * ctl[p].h);
  lam[2 * p] = L;
  lam[2 * p + 1] = L;
}

__global__ void berror_kernel(const double* __restrict__ y, const double* __restrict__ ynew,
                              Combo ce, FlowCtl* __restrict__ ctl, const Seg* __restrict__ seg,
                              const int* __restrict__ prefix, int n) {
  const int p = point_of(prefix, n, blockIdx.x);
  FlowCtl& c = ctl[p];
  if (c.done) return;  // uniform over the CTA
  const double h = c.h, rtol = c.rtol, atol = c.atol;
  const long long b = seg[p].off + (long long)(blockIdx.x - prefix[p]) * kChunk;
  const long long e = min(b + kChunk, seg[p].off + seg[p].len);
  unsigned long long emax = 0, ymax = 0;
  int bad = 0;
#pragma unroll
  for (int u = 0; u < kChunk / kFlowThreads; ++u) {
    const long long i = b + u * kFlowThreads + threadIdx.x;
    if (i >= e) break;
    const double acc = combo_sum(ce, i);
    const double yn = ynew[i];
    const double sc = atol + rtol * fmax(fabs(y[i]), fabs(yn));
    // the ratio in FP32 (the step control needs a few digits of it; GB300's
    // FP64 division costs more than the rest of the kernel)
    const double r = (double)__fdiv_rn((float)fabs(h * acc), (float)sc);
    if (!isfinite(yn) || !isfinite(r)) bad = 1;
    emax = max(emax, abs_bits(r));
    ymax = max(ymax, abs_bits(yn));
  }
  if (bad) c.nonfinite = 1;
  block_max_u(emax, &c.err_u);
  block_max_u(ymax, &c.max_u);
}

__global__ void bcontrol_kernel(FlowCtl* __restrict__ ctl, int* __restrict__ skip, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  FlowCtl* c = ctl + p;
  if (c->done) {
    c->accepted = 0;  // keeps the last step (dense output) intact
    skip[p] = 1;
    return;
  }
  control_update(c);
  skip[p] = c->done;
}

__global__ void baccept_kernel(double* __restrict__ y, const double* __restrict__ ynew,
                               double* __restrict__ yprev, double* __restrict__ k1,
                               const double* __restrict__ k7, double* __restrict__ k1prev,
                               const FlowCtl* __restrict__ ctl, const Seg* __restrict__ seg,
                               const int* __restrict__ prefix, int n) {
  const int p = point_of(prefix, n, blockIdx.x);
  if (!ctl[p].accepted) return;
  const long long b = seg[p].off + (long long)(blockIdx.x - prefix[p]) * kChunk;
  const long long e = min(b + kChunk, seg[p].off + seg[p].len);
#pragma unroll
  for (int u = 0; u < kChunk / kFlowThreads; ++u) {
    const long long i = b + u * kFlowThreads + threadIdx.x;
    if (i >= e) break;
    yprev[i] = y[i];
    y[i] = ynew[i];
    k1prev[i] = k1[i];
    k1[i] = k7[i];
  }
}

// Crossed points: max |interpolant| at the bisection midpoint (track) or the
// interpolant at bis_b written over y (final).
__global__ void bhermite_kernel(const double* __restrict__ y0, const double* __restrict__ f0,
                                double* __restrict__ y1, const double* __restrict__ f1,
                                FlowCtl* __restrict__ ctl, const Seg* __restrict__ seg,
                                const int* __restrict__ prefix, int n, int final_write) {
  const int p = point_of(prefix, n, blockIdx.x);
  FlowCtl& c = ctl[p];
  if (!c.crossed) return;
  const double s0 = c.s_prev, s1 = c.s;
  const double s = final_write ? c.bis_b : 0.5 * (c.bis_a + c.bis_b);
  const long long b = seg[p].off + (long long)(blockIdx.x - prefix[p]) * kChunk;
  const long long e = min(b + kChunk, seg[p].off + seg[p].len);
  unsigned long long m = 0;
#pragma unroll
  for (int u = 0; u < kChunk / kFlowThreads; ++u) {
    const long long i = b + u * kFlowThreads + threadIdx.x;
    if (i >= e) break;
    const double v = hermite(s0, y0[i], f0[i], s1, y1[i], f1[i], s);
    if (final_write)
      y1[i] = v;
    else
      m = max(m, abs_bits(v));
  }
  if (!final_write) block_max_u(m, &c.bis_u);
}

__global__ void bbisect_kernel(FlowCtl* __restrict__ ctl, int n, int phase) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  FlowCtl* c = ctl + p;
  if (phase == 3) {  // before the max / argmax of the final states
    c->max_u = 0;
    c->arg_u = ~0ull;
    return;
  }
  if (!c->crossed) return;
  if (phase == 0) {  // start: the crossing lies in [s, s_prev] (s < s_prev)
    c->bis_a = c->s_prev;
    c->bis_b = c->s;
    c->bis_u = 0;
  } else if (phase == 1) {
    const double m = 0.5 * (c->bis_a + c->bis_b);
    if (__longlong_as_double((long long)c->bis_u) > c->thr)
      c->bis_b = m;
    else
      c->bis_a = m;
    c->bis_u = 0;
  } else {  // done: the state now sits at bis_b
    c->s = c->bis_b;
  }
}

__global__ void bmax_kernel(const double* __restrict__ y, FlowCtl* __restrict__ ctl,
                            const Seg* __restrict__ seg, const int* __restrict__ prefix, int n,
                            int arg) {
  const int p = point_of(prefix, n, blockIdx.x);
  FlowCtl& c = ctl[p];
  const long long b = seg[p].off + (long long)(blockIdx.x - prefix[p]) * kChunk;
  const long long e = min(b + kChunk, seg[p].off + seg[p].len);
  if (arg) {
    const unsigned long long target = c.max_u;
#pragma unroll
    for (int u = 0; u < kChunk / kFlowThreads; ++u) {
      const long long i = b + u * kFlowThreads + threadIdx.x;
      if (i >= e) break;
      if (abs_bits(y[i]) == target) atomicMin(&c.arg_u, (unsigned long long)(i - seg[p].off));
    }
    return;
  }
  unsigned long long m = 0;
#pragma unroll
  for (int u = 0; u < kChunk / kFlowThreads; ++u) {
    const long long i = b + u * kFlowThreads + threadIdx.x;
    if (i >= e) break;
    m = max(m, abs_bits(y[i]));
  }
  block_max_u(m, &c.max_u);
}

}  // namespace

// Batch flow buffers and state (host side of tufrg_batch_flow).
struct BatchFlow {
  size_t n_state = 0;
  double* base = nullptr;
  double *y, *k[7], *ytmp, *ynew, *yprev, *k1prev;
  FlowCtl* ctl = nullptr;   // device [n]
  FlowCtl* hctl = nullptr;  // pinned host mirror
  // segments of the packed vectors and chunks per point, for the full
  // states [0] and the wedge layout [1]; seg, prefix, n_chunks: the layout
  // the flow integrates
  Seg* seg_lay[2] = {nullptr, nullptr};
  int* prefix_lay[2] = {nullptr, nullptr};
  int n_chunks_lay[2] = {0, 0};
  Seg* seg = nullptr;
  int* prefix = nullptr;
  int n_chunks = 0;
  cudaGraphExec_t attempt = nullptr;
  // every point's state is point-group covariant (checked at the start):
  // the flow integrates the states at the rows' representative l only
  // (wedge layout); the attempt graph was captured with graph_wedge
  bool wedge = false, graph_wedge = false;
  unsigned long long* cov = nullptr;  // device [2 n]: deviation, max |y| per point
};

}  // namespace tufrg

struct tufrg_batch {
  int n = 0;
  int precision = TUFRG_BF16X3;
  std::vector<tufrg_ctx*> pts;
  tufrg::MultiView view;
  double* d_lam = nullptr;  // [n][2]
  int* d_skip = nullptr;    // [n]
  int* d_err = nullptr;
  double* d_chi = nullptr;
  double* d_V = nullptr;    // couplings (FP32, the batch's arithmetic)
  float* d_y32 = nullptr;   // FP32 copy of the state for the projections
  double2* d_bt = nullptr;
  double2* d_fkey = nullptr;
  std::vector<long long> loop_off;
  tufrg::BatchFlow flow;
  cudaStream_t fstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaStream_t pstream = nullptr;  // projections beside the loops
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_stage = nullptr;
};

namespace tufrg {
namespace {

int grid_for(int n) { return (n + 127) / 128; }

// wedge: y and dy in the wedge layout (flows of point-group covariant
// states), projections and products at the rows' representative l only
// y32: the FP32 copy of y already written on b->pstream, or null (made here)
tufrg_status batch_rhs_device(tufrg_batch* b, const double* y, double* dy, bool scaled,
                              cudaStream_t st, bool wedge = false, const float* y32 = nullptr) {
  const MultiView& v = b->view;
  // the projections (states only) beside the loops (scales only)
  TUFRG_CUDA(cudaEventRecord(b->ev_fork, st));
  TUFRG_CUDA(cudaStreamWaitEvent(b->pstream, b->ev_fork, 0));
  if (!y32) {
    TUFRG_CHECK(launch_to_f32(y, b->d_y32, wedge ? v.wstate_elems : v.state_elems, b->pstream));
    y32 = b->d_y32;
  }
  TUFRG_CHECK(launch_project_multi(v, b->precision, y32, b->d_V, b->d_bt, b->d_fkey, b->pstream,
                                   wedge));
  TUFRG_CUDA(cudaEventRecord(b->ev_join, b->pstream));
  TUFRG_CHECK(launch_loops_tc_rows_multi(v, st));  // row loops, gathered by the products
  TUFRG_CUDA(cudaStreamWaitEvent(st, b->ev_join, 0));
  return launch_products_multi(v, b->precision, b->d_V, nullptr, dy, scaled, st, wedge);
}

tufrg_status set_lambdas(tufrg_batch* b, const double* lambda, cudaStream_t st) {
  std::vector<double> h(2 * (size_t)b->n);
  for (int i = 0; i < b->n; ++i) {
    if (!(std::isfinite(lambda[i]) && lambda[i] > 0.0)) return TUFRG_ERR_ARG;
    h[2 * i] = h[2 * i + 1] = lambda[i];
  }
  TUFRG_CUDA(cudaMemcpyAsync(b->d_lam, h.data(), sizeof(double) * h.size(),
                             cudaMemcpyHostToDevice, st));
  TUFRG_CUDA(cudaMemsetAsync(b->d_skip, 0, sizeof(int) * b->n, st));
  return TUFRG_OK;  // (a copy from pageable memory returns once h is staged)
}

void free_batch_flow(BatchFlow& f) {
  if (f.attempt) cudaGraphExecDestroy(f.attempt);
  void* ptrs[] = {f.base, f.seg_lay[0], f.prefix_lay[0]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (f.hctl) cudaFreeHost(f.hctl);
  f = BatchFlow();
}

tufrg_status batch_flow_buffers(tufrg_batch* b) {
  BatchFlow& f = b->flow;
  if (f.base) return TUFRG_OK;
  const size_t n = b->view.state_elems;
  f.n_state = n;
  const size_t bytes =
      sizeof(double) * n * 12 + sizeof(FlowCtl) * b->n + 256 + 16 * (size_t)b->n + 256;
  if (cudaMalloc((void**)&f.base, bytes) != cudaSuccess) return TUFRG_ERR_OOM;
  double* p = f.base;
  f.y = p;
  for (int i = 0; i < 7; ++i) f.k[i] = p + n * (1 + i);
  f.ytmp = p + n * 8;
  f.ynew = p + n * 9;
  f.yprev = p + n * 10;
  f.k1prev = p + n * 11;
  f.ctl = reinterpret_cast<FlowCtl*>(p + n * 12);
  f.cov = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(f.ctl + b->n) + 255) & ~uintptr_t(255));
  TUFRG_CUDA(cudaMallocHost((void**)&f.hctl, sizeof(FlowCtl) * b->n));
  std::vector<Seg> seg(2 * (size_t)b->n);
  std::vector<int> prefix(2 * (size_t)(b->n + 1), 0);
  for (int w = 0; w < 2; ++w)
    for (int i = 0; i < b->n; ++i) {
      const PointDesc& d = b->view.h[i];
      Seg& g = seg[(size_t)w * b->n + i];
      g.off = w ? d.off_wstate : d.off_state;
      g.len = 3LL * (w ? d.nrow : d.nl) * d.nff * d.nff;
      int* pf = prefix.data() + (size_t)w * (b->n + 1);
      pf[i + 1] = pf[i] + (int)((g.len + kChunk - 1) / kChunk);
    }
  if (cudaMalloc((void**)&f.seg_lay[0], sizeof(Seg) * seg.size()) != cudaSuccess ||
      cudaMalloc((void**)&f.prefix_lay[0], sizeof(int) * prefix.size()) != cudaSuccess)
    return TUFRG_ERR_OOM;
  f.seg_lay[1] = f.seg_lay[0] + b->n;
  f.prefix_lay[1] = f.prefix_lay[0] + (b->n + 1);
  for (int w = 0; w < 2; ++w) f.n_chunks_lay[w] = prefix[(size_t)w * (b->n + 1) + b->n];
  TUFRG_CUDA(cudaMemcpy(f.seg_lay[0], seg.data(), sizeof(Seg) * seg.size(),
                        cudaMemcpyHostToDevice));
  TUFRG_CUDA(cudaMemcpy(f.prefix_lay[0], prefix.data(), sizeof(int) * prefix.size(),
                        cudaMemcpyHostToDevice));
  return TUFRG_OK;
}

tufrg_status bstage(tufrg_batch* b, const double* y, double* out,
                    const std::vector<std::pair<double, const double*>>& terms, double cnode,
                    double* k_out, cudaStream_t st) {
  BatchFlow& f = b->flow;
  Combo cb{};
  cb.nk = (int)terms.size();
  for (int j = 0; j < cb.nk; ++j) {
    cb.a[j] = terms[j].first;
    cb.k[j] = terms[j].second;
  }
  cb.c = cnode;
  // the stage's states on the projection stream, the scales on the loop stream
  TUFRG_CUDA(cudaEventRecord(b->ev_stage, st));
  TUFRG_CUDA(cudaStreamWaitEvent(b->pstream, b->ev_stage, 0));
  bcombo_kernel<<<f.n_chunks, kFlowThreads, 0, b->pstream>>>(y, out, cb, f.ctl, b->d_lam, f.seg,
                                                             f.prefix, b->n, 0, b->d_y32);
  bstage_lambda_kernel<<<grid_for(b->n), 128, 0, st>>>(f.ctl, cnode, b->d_lam, b->n);
  TUFRG_CUDA(cudaGetLastError());
  return batch_rhs_device(b, out, k_out, true, st, f.wedge, b->d_y32);
}

tufrg_status enqueue_battempt(tufrg_batch* b, cudaStream_t st) {
  BatchFlow& f = b->flow;
  for (int i = 1; i < 7; ++i) {
    std::vector<std::pair<double, const double*>> t;
    for (int j = 0; j < i; ++j)
      if (kA[i][j] != 0.0) t.push_back({kA[i][j], f.k[j]});
    TUFRG_CHECK(bstage(b, f.y, i == 6 ? f.ynew : f.ytmp, t, kC[i], f.k[i], st));
  }
  Combo ce{};
  for (int j = 0; j < 7; ++j)
    if (kB[j] != kBs[j]) {
      ce.a[ce.nk] = kB[j] - kBs[j];
      ce.k[ce.nk] = f.k[j];
      ++ce.nk;
    }
  berror_kernel<<<f.n_chunks, kFlowThreads, 0, st>>>(f.y, f.ynew, ce, f.ctl, f.seg, f.prefix,
                                                     b->n);
  bcontrol_kernel<<<grid_for(b->n), 128, 0, st>>>(f.ctl, b->d_skip, b->n);
  baccept_kernel<<<f.n_chunks, kFlowThreads, 0, st>>>(f.y, f.ynew, f.yprev, f.k[0], f.k[6],
                                                      f.k1prev, f.ctl, f.seg, f.prefix, b->n);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status battempt_graph(tufrg_batch* b, cudaStream_t st) {
  BatchFlow& f = b->flow;
  if (f.attempt) return TUFRG_OK;
  cudaGraph_t g = nullptr;
  TUFRG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  tufrg_status s = enqueue_battempt(b, st);
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (s != TUFRG_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  TUFRG_CUDA(e);
  e = cudaGraphInstantiate(&f.attempt, g, 0);
  cudaGraphDestroy(g);
  TUFRG_CUDA(e);
  return TUFRG_OK;
}

tufrg_status read_ctls(tufrg_batch* b, cudaStream_t st) {
  BatchFlow& f = b->flow;
  TUFRG_CUDA(cudaMemcpyAsync(f.hctl, f.ctl, sizeof(FlowCtl) * b->n, cudaMemcpyDeviceToHost, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

tufrg_status check_err(int* d_err, cudaStream_t st) {
  int err = 0;
  TUFRG_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  if (err) {
    TUFRG_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    TUFRG_CUDA(cudaStreamSynchronize(st));
    return TUFRG_ERR_TIMEOUT;
  }
  return TUFRG_OK;
}

tufrg_status batch_flow(tufrg_batch* b, const tufrg_flow_opts* o, double* y_dev,
                        tufrg_result* res, int32_t* status, cudaStream_t st) {
  TUFRG_CHECK(batch_flow_buffers(b));
  BatchFlow& f = b->flow;
  const size_t n = f.n_state;
  const int np = b->n;
  std::vector<FlowCtl> h0(np);
  for (int i = 0; i < np; ++i) {
    FlowCtl& c = h0[i];
    c = FlowCtl{};
    c.s = std::log(o->lambda0);
    c.s_end = std::log(o->lambda_min);
    c.dir = -1.0;
    c.rtol = o->rtol;
    c.atol = o->atol;
    c.thr = o->threshold;
    c.h = -std::fabs(o->h0);
    if (c.s + c.h < c.s_end) c.h = c.s_end - c.s;
  }
  std::memcpy(f.hctl, h0.data(), sizeof(FlowCtl) * np);
  TUFRG_CUDA(cudaMemcpyAsync(f.ctl, f.hctl, sizeof(FlowCtl) * np, cudaMemcpyHostToDevice, st));
  TUFRG_CUDA(cudaMemsetAsync(b->d_skip, 0, sizeof(int) * np, st));
  TUFRG_CUDA(cudaMemcpyAsync(f.y, y_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  // the wedge when every point's initial state is covariant (zeros are)
  {
    TUFRG_CHECK(launch_covariance_check(b->view, f.y, f.cov, st));
    std::vector<unsigned long long> h(2 * (size_t)np);
    TUFRG_CUDA(cudaMemcpyAsync(h.data(), f.cov, sizeof(unsigned long long) * h.size(),
                               cudaMemcpyDeviceToHost, st));
    TUFRG_CUDA(cudaStreamSynchronize(st));
    f.wedge = true;
    for (int i = 0; i < np; ++i) {
      double dev, amax;
      std::memcpy(&dev, &h[2 * i], 8);
      std::memcpy(&amax, &h[2 * i + 1], 8);
      f.wedge = f.wedge && dev <= 1e-13 * amax;
    }
    if (f.wedge != f.graph_wedge && f.attempt) {
      cudaGraphExecDestroy(f.attempt);
      f.attempt = nullptr;
    }
    f.graph_wedge = f.wedge;
  }
  const int lay = f.wedge ? 1 : 0;
  f.seg = f.seg_lay[lay];
  f.prefix = f.prefix_lay[lay];
  f.n_chunks = f.n_chunks_lay[lay];
  if (f.wedge) {
    TUFRG_CHECK(launch_wedge_compress(b->view, f.y, f.ynew, st));
    TUFRG_CUDA(cudaMemcpyAsync(f.y, f.ynew, sizeof(double) * b->view.wstate_elems,
                               cudaMemcpyDeviceToDevice, st));
  }
  TUFRG_CHECK(bstage(b, f.y, f.ytmp, {}, 0.0, f.k[0], st));  // k1 = f(s0, y0)
  TUFRG_CHECK(battempt_graph(b, st));
  int attempts = 0;
  for (; attempts < o->max_steps; ++attempts) {
    TUFRG_CUDA(cudaGraphLaunch(f.attempt, st));
    TUFRG_CHECK(read_ctls(b, st));
    bool all = true;
    for (int i = 0; i < np && all; ++i) all = f.hctl[i].done != 0;
    if (all) break;
  }
  // crossings: bisection on the interpolants of the crossed points' last steps
  const int G = grid_for(np);
  bbisect_kernel<<<G, 128, 0, st>>>(f.ctl, np, 0);
  for (int it = 0; it < kBisect; ++it) {
    bhermite_kernel<<<f.n_chunks, kFlowThreads, 0, st>>>(f.yprev, f.k1prev, f.y, f.k[0], f.ctl,
                                                         f.seg, f.prefix, np, 0);
    bbisect_kernel<<<G, 128, 0, st>>>(f.ctl, np, 1);
  }
  bhermite_kernel<<<f.n_chunks, kFlowThreads, 0, st>>>(f.yprev, f.k1prev, f.y, f.k[0], f.ctl,
                                                       f.seg, f.prefix, np, 1);
  bbisect_kernel<<<G, 128, 0, st>>>(f.ctl, np, 2);
  bbisect_kernel<<<G, 128, 0, st>>>(f.ctl, np, 3);
  // the final states in full (wedge layouts expanded to every l), then their
  // largest elements
  if (f.wedge)
    TUFRG_CHECK(launch_wedge_expand(b->view, f.y, y_dev, st));
  else
    TUFRG_CUDA(cudaMemcpyAsync(y_dev, f.y, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  bmax_kernel<<<f.n_chunks_lay[0], kFlowThreads, 0, st>>>(y_dev, f.ctl, f.seg_lay[0],
                                                          f.prefix_lay[0], np, 0);
  bmax_kernel<<<f.n_chunks_lay[0], kFlowThreads, 0, st>>>(y_dev, f.ctl, f.seg_lay[0],
                                                          f.prefix_lay[0], np, 1);
  TUFRG_CUDA(cudaGetLastError());
  TUFRG_CHECK(read_ctls(b, st));
  tufrg_status first = TUFRG_OK;
  for (int i = 0; i < np; ++i) {
    const FlowCtl& c = f.hctl[i];
    tufrg_result& r = res[i];
    r = tufrg_result{};
    r.lambda_c = std::exp(c.s);
    r.h_next = std::fabs(c.h);
    r.diverged = c.crossed ? 1 : 0;
    r.finished = c.done ? 1 : 0;
    r.n_accepted = c.n_acc;
    r.n_rejected = c.n_rej;
    r.n_rhs = 1 + c.n_rhs;
    double mx;
    std::memcpy(&mx, &c.max_u, sizeof mx);
    r.max_abs = mx;
    const PointDesc& d = b->view.h[i];
    const long long per_ch = (long long)d.nl * d.nff * d.nff;
    const unsigned long long idx = c.arg_u;
    if (idx < (unsigned long long)(3 * per_ch)) {
      r.channel = (int32_t)(idx / per_ch);
      long long rem = (long long)(idx % per_ch);
      r.l_index = (int32_t)(rem / ((long long)d.nff * d.nff));
      rem %= (long long)d.nff * d.nff;
      r.m = (int32_t)(rem / d.nff);
      r.n = (int32_t)(rem % d.nff);
    } else {
      r.channel = r.l_index = r.m = r.n = -1;
    }
    if (status) status[i] = c.status;
    if (c.status != TUFRG_OK && first == TUFRG_OK) first = (tufrg_status)c.status;
  }
  const tufrg_status e = check_err(b->d_err, st);
  return first != TUFRG_OK ? first : e;
}

// the candidates: the default, and a ladder around it within the chain cap
std::vector<int> tune_candidates(const MultiView& v) {
  const int d = view_default_kbps(v);
  const int cap = max_kbps(v.tc_prec);
  std::vector<int> c = {d};
  for (int k : {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256})
    if (k <= cap) c.push_back(k);
  std::sort(c.begin(), c.end());
  c.erase(std::unique(c.begin(), c.end()), c.end());
  if (c.size() > 16) c.resize(16);
  return c;
}

struct CtxRun {
  tufrg_ctx* c;
  double lambda;
};
tufrg_status run_ctx(void* arg, cudaStream_t st) {
  CtxRun* r = static_cast<CtxRun*>(arg);
  TUFRG_CHECK(launch_set_scalar(r->c->d_lambda, r->lambda, st));
  return launch_loops_tc_multi(r->c->view, r->c->d_chi, st);
}

tufrg_status run_batch(void* arg, cudaStream_t st) {
  tufrg_batch* b = static_cast<tufrg_batch*>(arg);
  return launch_loops_tc_multi(b->view, b->d_chi, st);
}

}  // namespace

tufrg_status autotune_view(MultiView& v, tufrg_status (*run)(void*, cudaStream_t), void* arg,
                           tufrg_tune_report* rep, cudaStream_t st) {
  if (v.tc_prec == TUFRG_FP64) return TUFRG_ERR_ARG;
  const std::vector<int> cand = tune_candidates(v);
  cudaEvent_t e0, e1;
  TUFRG_CUDA(cudaEventCreate(&e0));
  TUFRG_CUDA(cudaEventCreate(&e1));
  std::vector<double> ms(cand.size(), 0.0);
  tufrg_status s = TUFRG_OK;
  for (size_t i = 0; i < cand.size() && s == TUFRG_OK; ++i) {
    s = view_set_kbps(v, cand[i], st);
    if (s == TUFRG_OK) s = run(arg, st);  // warm-up
    float t[3] = {0, 0, 0};
    for (int r = 0; r < 3 && s == TUFRG_OK; ++r) {
      if (cudaEventRecord(e0, st) != cudaSuccess) s = TUFRG_ERR_CUDA;
      if (s == TUFRG_OK) s = run(arg, st);
      if (s == TUFRG_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                            cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess))
        s = TUFRG_ERR_CUDA;
    }
    std::sort(t, t + 3);
    ms[i] = t[1];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TUFRG_CHECK(s);
  const size_t best = std::min_element(ms.begin(), ms.end()) - ms.begin();
  TUFRG_CHECK(view_set_kbps(v, cand[best], st));
  if (rep) {
    *rep = tufrg_tune_report{};
    rep->n_candidates = (int32_t)cand.size();
    for (size_t i = 0; i < cand.size(); ++i) {
      rep->kbps[i] = cand[i];
      rep->ms[i] = ms[i];
    }
    rep->chosen = (int32_t)best;
    rep->kbps_default = view_default_kbps(v);
  }
  return TUFRG_OK;
}

}  // namespace tufrg

using tufrg::BatchFlow;

namespace {

void batch_free(tufrg_batch* b) {
  cudaDeviceSynchronize();
  tufrg::free_batch_flow(b->flow);
  tufrg::view_free(b->view);
  void* ptrs[] = {b->d_lam, b->d_skip, b->d_err, b->d_chi, b->d_V, b->d_bt, b->d_fkey, b->d_y32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (tufrg_ctx* c : b->pts)
    if (c) {
      tufrg::free_device(c);
      delete c;
    }
  for (cudaEvent_t e : {b->ev_in, b->ev_out, b->ev_fork, b->ev_join, b->ev_stage})
    if (e) cudaEventDestroy(e);
  for (cudaStream_t q : {b->fstream, b->pstream})
    if (q) cudaStreamDestroy(q);
  delete b;
}

tufrg_status batch_setup(int32_t n, const tufrg_params* params, cudaStream_t st,
                         tufrg_batch* b) {
  b->n = n;
  b->precision = params[0].precision;
  if (b->precision == TUFRG_FP64) return TUFRG_ERR_ARG;  // batches run the tensor-core loops
  b->pts.assign(n, nullptr);
  // donors of shared tables: first point with the same key
  using Bonds = std::vector<int32_t>;
  std::map<std::tuple<int, int, int, int, Bonds>, int> loops_key;
  std::map<std::tuple<int, int, Bonds>, int> proj_key;
  for (int i = 0; i < n; ++i) {
    const tufrg_params& p = params[i];
    if (p.precision != b->precision || p.n_bonds < 0 || (p.n_bonds > 0 && !p.bonds))
      return TUFRG_ERR_ARG;
    Bonds bonds(p.bonds, p.bonds + 2 * p.n_bonds);
    auto lk = std::make_tuple(p.nf_x, p.nf_y, p.nc_x, p.nc_y, bonds);
    auto pk = std::make_tuple(p.nc_x, p.nc_y, bonds);
    tufrg::SetupShare share;
    share.own_view = false;
    share.workspace = false;
    auto li = loops_key.find(lk);
    if (li != loops_key.end()) share.loops = b->pts[li->second];
    auto pi = proj_key.find(pk);
    if (pi != proj_key.end()) share.proj = b->pts[pi->second];
    TUFRG_CHECK(tufrg::create_context(&p, st, share, &b->pts[i]));
    if (li == loops_key.end()) loops_key.emplace(lk, i);
    if (pi == proj_key.end()) proj_key.emplace(pk, i);
  }
  if (cudaMalloc((void**)&b->d_lam, sizeof(double) * 2 * n) != cudaSuccess ||
      cudaMalloc((void**)&b->d_skip, sizeof(int) * n) != cudaSuccess ||
      cudaMalloc((void**)&b->d_err, sizeof(int)) != cudaSuccess)
    return TUFRG_ERR_OOM;
  TUFRG_CUDA(cudaMemsetAsync(b->d_skip, 0, sizeof(int) * n, st));
  TUFRG_CUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), st));
  std::vector<double*> lam(n);
  std::vector<const int*> skip(n);
  for (int i = 0; i < n; ++i) {
    lam[i] = b->d_lam + 2 * i;
    skip[i] = b->d_skip + i;
  }
  TUFRG_CHECK(tufrg::view_build(b->view, b->pts.data(), n, lam.data(), skip.data(), b->d_err,
                                b->precision, 0, st));
  const tufrg::MultiView& v = b->view;
  if (cudaMalloc((void**)&b->d_chi, sizeof(double) * std::max<size_t>(v.chi_elems, 1)) !=
          cudaSuccess ||
      cudaMalloc((void**)&b->d_V, sizeof(double) * std::max<size_t>(v.state_elems, 1)) !=
          cudaSuccess ||
      cudaMalloc((void**)&b->d_y32, sizeof(float) * std::max<size_t>(v.state_elems, 1)) !=
          cudaSuccess ||
      cudaMalloc((void**)&b->d_bt, sizeof(double2) * std::max<size_t>(v.bt_elems, 1)) !=
          cudaSuccess ||
      cudaMalloc((void**)&b->d_fkey, sizeof(double2) * std::max<size_t>(v.fkey_elems, 1)) !=
          cudaSuccess)
    return TUFRG_ERR_OOM;
  TUFRG_CUDA(cudaMemsetAsync(b->d_chi, 0, sizeof(double) * v.chi_elems, st));
  TUFRG_CUDA(cudaStreamCreateWithFlags(&b->fstream, cudaStreamNonBlocking));
  TUFRG_CUDA(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
  TUFRG_CUDA(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  TUFRG_CUDA(cudaStreamCreateWithFlags(&b->pstream, cudaStreamNonBlocking));
  TUFRG_CUDA(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  TUFRG_CUDA(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
  TUFRG_CUDA(cudaEventCreateWithFlags(&b->ev_stage, cudaEventDisableTiming));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  return TUFRG_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

extern "C" {

tufrg_status tufrg_batch_setup(int32_t n_points, const tufrg_params* params, void* cuda_stream,
                               tufrg_batch** out) {
  if (!out) return TUFRG_ERR_ARG;
  *out = nullptr;
  if (n_points < 1 || !params) return TUFRG_ERR_ARG;
  tufrg_batch* b = new (std::nothrow) tufrg_batch();
  if (!b) return TUFRG_ERR_OOM;
  const tufrg_status s = batch_setup(n_points, params, (cudaStream_t)cuda_stream, b);
  if (s != TUFRG_OK) {
    batch_free(b);
    return s;
  }
  *out = b;
  return TUFRG_OK;
}

void tufrg_batch_destroy(tufrg_batch* b) {
  if (b) batch_free(b);
}

tufrg_status tufrg_batch_dims(const tufrg_batch* b, int32_t point, int32_t* nl, int32_t* nff,
                              int64_t* state_offset, int64_t* loop_offset) {
  if (!b || point < -1 || point >= b->n) return TUFRG_ERR_ARG;
  if (point == -1) {
    if (nl) *nl = b->n;
    if (nff) *nff = b->view.nff_max;
    if (state_offset) *state_offset = (int64_t)b->view.state_elems;
    if (loop_offset) *loop_offset = (int64_t)b->view.chi_elems;
    return TUFRG_OK;
  }
  const tufrg::PointDesc& d = b->view.h[point];
  if (nl) *nl = d.nl;
  if (nff) *nff = d.nff;
  if (state_offset) *state_offset = d.off_state;
  if (loop_offset) *loop_offset = d.off_chi;
  return TUFRG_OK;
}

tufrg_status tufrg_batch_loops(tufrg_batch* b, const double* lambda, double* chi_dot_dev,
                               void* cuda_stream) {
  if (!b || !lambda || !chi_dot_dev) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TUFRG_CHECK(tufrg::set_lambdas(b, lambda, st));
  return tufrg::launch_loops_tc_multi(b->view, chi_dot_dev, st);
}

tufrg_status tufrg_batch_rhs(tufrg_batch* b, const double* lambda, const double* y_dev,
                             double* dy_dev, void* cuda_stream) {
  if (!b || !lambda || !y_dev || !dy_dev || y_dev == dy_dev) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TUFRG_CHECK(tufrg::set_lambdas(b, lambda, st));
  return tufrg::batch_rhs_device(b, y_dev, dy_dev, false, st);
}

tufrg_status tufrg_batch_flow(tufrg_batch* b, const tufrg_flow_opts* o, double* y_dev,
                              tufrg_result* res, int32_t* status, void* cuda_stream) {
  if (!b || !o || !y_dev || !res || o->max_steps <= 0) return TUFRG_ERR_ARG;
  if (!finite_pos(o->lambda0) || !finite_pos(o->lambda_min) || o->lambda_min >= o->lambda0 ||
      !finite_pos(o->threshold) || !(o->rtol >= 0.0) || !(o->atol >= 0.0) ||
      o->rtol + o->atol <= 0.0 || !finite_pos(o->h0) || o->method != TUFRG_DOPRI5 ||
      o->n_checkpoints != 0 || o->fp64_above != 0.0)
    return TUFRG_ERR_ARG;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  TUFRG_CUDA(cudaEventRecord(b->ev_in, user));
  TUFRG_CUDA(cudaStreamWaitEvent(b->fstream, b->ev_in, 0));
  const tufrg_status s = tufrg::batch_flow(b, o, y_dev, res, status, b->fstream);
  if (cudaEventRecord(b->ev_out, b->fstream) != cudaSuccess ||
      cudaStreamWaitEvent(user, b->ev_out, 0) != cudaSuccess)
    return s == TUFRG_OK ? TUFRG_ERR_CUDA : s;
  return s;
}

tufrg_status tufrg_batch_autotune(tufrg_batch* b, double lambda, tufrg_tune_report* rep,
                                  void* cuda_stream) {
  if (!b || !finite_pos(lambda)) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::vector<double> lam(b->n, lambda);
  TUFRG_CHECK(tufrg::set_lambdas(b, lam.data(), st));
  if (b->flow.attempt) {  // the work items change: recapture on the next flow
    cudaGraphExecDestroy(b->flow.attempt);
    b->flow.attempt = nullptr;
  }
  TUFRG_CHECK(tufrg::autotune_view(b->view, tufrg::run_batch, b, rep, st));
  return tufrg::check_err(b->d_err, st);
}

tufrg_status tufrg_autotune(tufrg_ctx* c, double lambda, tufrg_tune_report* rep,
                            void* cuda_stream) {
  if (!c || !finite_pos(lambda) || c->p.precision == TUFRG_FP64) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  tufrg::flow_drop_graphs(c);
  tufrg::CtxRun r{c, lambda};
  TUFRG_CHECK(tufrg::autotune_view(c->view, tufrg::run_ctx, &r, rep, st));
  return tufrg::check_err(c->d_err, st);
}

tufrg_status tufrg_batch_profile_loops(tufrg_batch* b, double lambda, int32_t n,
                                       double* kernel_ms, double* stage_ms, void* cuda_stream) {
  if (!b || n < 1 || !finite_pos(lambda) || !kernel_ms || !stage_ms) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::vector<double> lam(b->n, lambda);
  TUFRG_CHECK(tufrg::set_lambdas(b, lam.data(), st));
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  tufrg_status s = TUFRG_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) s = TUFRG_ERR_CUDA;
  double k = 0.0, g = 0.0;
  for (int i = 0; i < n && s == TUFRG_OK; ++i) {
    if (cudaEventRecord(ev[2], st) != cudaSuccess) s = TUFRG_ERR_CUDA;
    if (s == TUFRG_OK) s = tufrg::launch_loops_tc_rows_multi(b->view, st, ev);
    if (s == TUFRG_OK && cudaEventRecord(ev[3], st) != cudaSuccess) s = TUFRG_ERR_CUDA;
    float a = 0.f, c = 0.f;
    if (s == TUFRG_OK &&
        (cudaEventSynchronize(ev[3]) != cudaSuccess ||
         cudaEventElapsedTime(&a, ev[0], ev[1]) != cudaSuccess ||
         cudaEventElapsedTime(&c, ev[2], ev[3]) != cudaSuccess))
      s = TUFRG_ERR_CUDA;
    k += a;
    g += c;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  TUFRG_CHECK(s);
  *kernel_ms = k / n;
  *stage_ms = g / n;
  return tufrg::check_err(b->d_err, st);
}

tufrg_status tufrg_batch_check(tufrg_batch* b, void* cuda_stream) {
  if (!b) return TUFRG_ERR_ARG;
  return tufrg::check_err(b->d_err, (cudaStream_t)cuda_stream);
}

}  // extern "C"
