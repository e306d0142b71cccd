// extern "C" entry points of include/tufrg.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

namespace {
thread_local cudaError_t g_last_cuda_error = cudaSuccess;
thread_local char g_last_cuda_where[160] = "";
}

tufrg_status tufrg_cuda_fail(cudaError_t e) {
  g_last_cuda_error = e;
  g_last_cuda_where[0] = 0;
  if (e == cudaErrorMemoryAllocation) return TUFRG_ERR_OOM;
  return TUFRG_ERR_CUDA;
}

tufrg_status tufrg_cuda_fail_at(cudaError_t e, const char* file, int line) {
  const tufrg_status s = tufrg_cuda_fail(e);
  const char* base = std::strrchr(file, '/');
  std::snprintf(g_last_cuda_where, sizeof g_last_cuda_where, "%s at %s:%d", cudaGetErrorName(e),
                base ? base + 1 : file, line);
  return s;
}

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

tufrg_status validate(const tufrg_params* p) {
  if (!p || p->lattice != 0) return TUFRG_ERR_ARG;
  if (!std::isfinite(p->t) || p->t == 0.0 || !std::isfinite(p->tp) || !std::isfinite(p->mu) ||
      !std::isfinite(p->U))
    return TUFRG_ERR_ARG;
  if (p->nc_x < 2 || p->nc_y < 2 || (p->nc_x & 1) || (p->nc_y & 1)) return TUFRG_ERR_ARG;
  if (p->nf_x < 4 || p->nf_y < 4) return TUFRG_ERR_ARG;
  // p +- l/2 on the fine grid (table mode) unless the loops are FP64, which
  // also evaluate xi there analytically
  if ((p->nf_x % (2 * p->nc_x) || p->nf_y % (2 * p->nc_y)) && p->precision != TUFRG_FP64)
    return TUFRG_ERR_ARG;
  if (p->nf_x % 4 || p->nf_y % 4) return TUFRG_ERR_ARG;
  if ((long long)p->nf_x * p->nf_y > (1LL << 26)) return TUFRG_ERR_ARG;
  if ((long long)p->nc_x * p->nc_y > (1LL << 16)) return TUFRG_ERR_ARG;
  if (p->precision < TUFRG_FP64 || p->precision > TUFRG_BF16X3) return TUFRG_ERR_ARG;
  if (p->feedback != 0 && p->feedback != 1) return TUFRG_ERR_ARG;
  return TUFRG_OK;
}

}  // namespace

namespace tufrg {

static bool sharded(const tufrg_ctx* c) { return c->shard_lo != 0 || c->shard_hi != c->nrow; }

tufrg_status launch_loops(tufrg_ctx* c, int prec, double* chi, cudaStream_t st) {
  if (sharded(c)) return TUFRG_ERR_STATE;  // the loops of every l need every row
  if (prec == kLoopSurrogate) {
    if (!c->sur || chi != c->d_chi) return TUFRG_ERR_STATE;
    return surrogate_loops(c->sur, c, chi, st);
  }
  // the row loops, their refinement correction, every l from the rows
  if (prec == TUFRG_FP64) {
    TUFRG_CHECK(launch_scale_tables(c, st));
    TUFRG_CHECK(launch_loops_fp64_rows(c, st));
  } else {
    TUFRG_CHECK(launch_loops_tc_rows_multi(c->view, st));
  }
  TUFRG_CHECK(launch_refine_rows(c, st));
  return launch_expand_multi(c->view, chi, st);
}

tufrg_status launch_loop_rows(tufrg_ctx* c, int prec, cudaStream_t st) {
  if (prec == kLoopSurrogate) return TUFRG_ERR_ARG;
  if (sharded(c)) return TUFRG_ERR_STATE;
  if (prec == TUFRG_FP64) {
    TUFRG_CHECK(launch_scale_tables(c, st));
    TUFRG_CHECK(launch_loops_fp64_rows(c, st));
  } else {
    TUFRG_CHECK(launch_loops_tc_rows_multi(c->view, st));
  }
  return launch_refine_rows(c, st);
}

int rhs_arith(const tufrg_ctx* c, int prec) {
  // projections and products in FP32 arithmetic for a mixed-precision
  // context, in FP64 for an FP64 context and after a switch to FP64 loops
  return (prec == TUFRG_FP64 || c->p.precision == TUFRG_FP64) ? TUFRG_FP64 : TUFRG_3XTF32;
}

tufrg_status rhs_device(tufrg_ctx* c, int prec, const double* y, double* dy, bool scaled,
                        cudaStream_t st, bool wedge, const float* y32) {
  const int arith = rhs_arith(c, prec);
  // the projections (state only) beside the loops (scale only)
  TUFRG_CUDA(cudaEventRecord(c->ev_fork, st));
  TUFRG_CUDA(cudaStreamWaitEvent(c->pstream, c->ev_fork, 0));
  // exact loops stay as row loops; the products gather each l from its row
  // (or, for a covariant state, run at the rows' representatives only)
  const bool rows = prec != kLoopSurrogate;
  if (wedge && !rows) return TUFRG_ERR_STATE;  // a wedge-layout state needs exact loops
  const void* yin = y;
  if (arith != TUFRG_FP64) {  // the FP32 kernels read an FP32 copy of the state
    if (!y32) {
      TUFRG_CHECK(launch_to_f32(y, c->d_y32, wedge ? c->view.wstate_elems : c->view.state_elems,
                                c->pstream));
      y32 = c->d_y32;
    }
    yin = y32;
  }
  TUFRG_CHECK(launch_project_multi(c->view, arith, yin, c->d_V, c->d_bt, c->d_fkey, c->pstream,
                                   wedge));
  TUFRG_CUDA(cudaEventRecord(c->ev_join, c->pstream));
  if (rows)
    TUFRG_CHECK(launch_loop_rows(c, prec, st));
  else
    TUFRG_CHECK(launch_loops(c, prec, c->d_chi, st));
  TUFRG_CUDA(cudaStreamWaitEvent(st, c->ev_join, 0));
  return launch_products_multi(c->view, arith, c->d_V, rows ? nullptr : c->d_chi, dy, scaled, st,
                               wedge);
}

tufrg_status create_context(const tufrg_params* p, cudaStream_t st, const SetupShare& share,
                            tufrg_ctx** out) {
  *out = nullptr;
  TUFRG_CHECK(validate(p));
  tufrg_ctx* c = new (std::nothrow) tufrg_ctx();
  if (!c) return TUFRG_ERR_OOM;
  c->p = *p;
  if (p->n_bonds > 0 && p->bonds) c->bonds.assign(p->bonds, p->bonds + 2 * p->n_bonds);
  c->p.bonds = c->bonds.data();
  tufrg_status s = c->basis.build(p->n_bonds, p->bonds);
  if (s == TUFRG_OK && (p->nc_x < 2 * c->basis.max_component + 1 ||
                        p->nc_y < 2 * c->basis.max_component + 1))
    s = TUFRG_ERR_ARG;  // coarse grid must resolve the basis
  if (s != TUFRG_OK) {
    delete c;
    return s;
  }
  c->ncx = p->nc_x;
  c->ncy = p->nc_y;
  c->nl = c->ncx * c->ncy;
  if (share.mesh) {
    c->mesh = true;
    c->mesh_m = share.mesh->m;
    c->mesh_pts = share.mesh->pts;
    c->mesh_w = share.mesh->w;
    c->nl = (int)c->mesh_pts.size();
  }
  c->nfx = p->nf_x;
  c->nfy = p->nf_y;
  c->nf = c->nfx * c->nfy;
  c->nff = c->basis.nff;
  c->nb = c->basis.nb;
  c->loop_prec = p->precision;
  s = setup_device(c, st, share);
  if (s != TUFRG_OK) {
    free_device(c);
    delete c;
    return s;
  }
  *out = c;
  return TUFRG_OK;
}

}  // namespace tufrg

extern "C" {

tufrg_status tufrg_setup(const tufrg_params* p, void* cuda_stream, tufrg_ctx** out) {
  if (!out) return TUFRG_ERR_ARG;
  *out = nullptr;
  return tufrg::create_context(p, (cudaStream_t)cuda_stream, tufrg::SetupShare(), out);
}

tufrg_status tufrg_setup_mesh(const tufrg_params* p, int32_t m, int32_t n_points,
                              const int32_t* points, const double* w_p, const double* w_cd,
                              void* cuda_stream, tufrg_ctx** out) {
  if (!out) return TUFRG_ERR_ARG;
  *out = nullptr;
  if (!p || !points || !w_p || !w_cd || p->nc_x != p->nc_y || m < 1 || m > 1023 || !(m & 1) ||
      n_points < 1 || n_points > (1 << 16))
    return TUFRG_ERR_ARG;
  const long long div = (long long)p->nc_x * m;
  if (div <= 0 || p->nf_x % (2 * div) || p->nf_y % (2 * div)) return TUFRG_ERR_ARG;
  tufrg::MeshSpec mesh;
  mesh.m = m;
  mesh.pts.resize(n_points);
  mesh.w.resize(2 * (size_t)n_points);
  double sum_p = 0.0, sum_cd = 0.0;
  std::vector<long long> keys(n_points);
  for (int i = 0; i < n_points; ++i) {
    const int jx = points[2 * i], jy = points[2 * i + 1];
    if (jx < 0 || jy < 0 || jx >= div || jy >= div) return TUFRG_ERR_ARG;
    const double a = w_p[i], b = w_cd[i];
    if (!std::isfinite(a) || !std::isfinite(b) || a < 0.0 || b < 0.0 || (a == 0.0 && b == 0.0))
      return TUFRG_ERR_ARG;  // every point belongs to one of the two meshes
    mesh.pts[i] = make_int2(jx, jy);
    mesh.w[i] = a;
    mesh.w[n_points + i] = b;
    sum_p += a;
    sum_cd += b;
    keys[i] = (long long)jx * div + jy;
  }
  if (std::fabs(sum_p - 1.0) > 1e-9 || std::fabs(sum_cd - 1.0) > 1e-9) return TUFRG_ERR_ARG;
  std::sort(keys.begin(), keys.end());
  if (std::adjacent_find(keys.begin(), keys.end()) != keys.end()) return TUFRG_ERR_ARG;
  tufrg::SetupShare share;
  share.mesh = &mesh;
  return tufrg::create_context(p, (cudaStream_t)cuda_stream, share, out);
}

void tufrg_destroy(tufrg_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  tufrg::free_device(c);
  delete c;
}

tufrg_status tufrg_dims(const tufrg_ctx* c, int32_t* nl, int32_t* nff, int32_t* nb) {
  if (!c) return TUFRG_ERR_ARG;
  if (nl) *nl = c->nl;
  if (nff) *nff = c->nff;
  if (nb) *nb = c->nb;
  return TUFRG_OK;
}

tufrg_status tufrg_eval_formfactors(int32_t n_bonds, const int32_t* bonds, int32_t n,
                                    const double* kx, const double* ky, double* out,
                                    int32_t* nff_out) {
  tufrg::Basis basis;
  TUFRG_CHECK(basis.build(n_bonds, bonds));
  if (nff_out) *nff_out = basis.nff;
  if (!out) return TUFRG_OK;
  if (n < 0 || (n > 0 && (!kx || !ky))) return TUFRG_ERR_ARG;
  for (int m = 0; m < basis.nff; ++m)
    for (int i = 0; i < n; ++i) out[(size_t)m * n + i] = basis.eval(m, kx[i], ky[i]);
  return TUFRG_OK;
}

tufrg_status tufrg_loops(tufrg_ctx* c, double lambda, double* chi_dot_dev, void* stream) {
  if (!c || !chi_dot_dev || !finite_pos(lambda)) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  TUFRG_CHECK(tufrg::launch_set_scalar(c->d_lambda, lambda, st));
  return tufrg::launch_loops(c, c->p.precision, chi_dot_dev, st);
}

tufrg_status tufrg_project(tufrg_ctx* c, const double* y_dev, double* v_dev, void* stream) {
  if (!c || !y_dev || !v_dev || y_dev == v_dev) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (c->p.precision == TUFRG_FP64)
    return tufrg::launch_project_multi(c->view, TUFRG_FP64, y_dev, v_dev, c->d_bt, c->d_fkey, st);
  // FP32 arithmetic on an FP32 copy of the state; the couplings returned in FP64
  const size_t n = c->view.state_elems;
  float* v32 = reinterpret_cast<float*>(c->d_V);
  TUFRG_CHECK(tufrg::launch_to_f32(y_dev, c->d_y32, n, st));
  TUFRG_CHECK(tufrg::launch_project_multi(c->view, c->p.precision, c->d_y32, v32, c->d_bt,
                                          c->d_fkey, st));
  return tufrg::launch_to_f64(v32, v_dev, n, st);
}

tufrg_status tufrg_products(tufrg_ctx* c, const double* v_dev, const double* chi_dot_dev,
                            double* dy_dev, void* stream) {
  if (!c || !v_dev || !chi_dot_dev || !dy_dev || dy_dev == v_dev || dy_dev == chi_dot_dev)
    return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (c->p.precision == TUFRG_FP64)
    return tufrg::launch_products_multi(c->view, TUFRG_FP64, v_dev, chi_dot_dev, dy_dev, false, st);
  // FP32 arithmetic on an FP32 copy of the couplings
  float* v32 = reinterpret_cast<float*>(c->d_V);
  TUFRG_CHECK(tufrg::launch_to_f32(v_dev, v32, c->view.state_elems, st));
  return tufrg::launch_products_multi(c->view, c->p.precision, v32, chi_dot_dev, dy_dev, false,
                                      st);
}

tufrg_status tufrg_set_refinement(tufrg_ctx* c, int32_t s, double kappa, double lambda_on,
                                  void* stream) {
  if (!c || !c->d_V) return TUFRG_ERR_ARG;
  if (c->mesh || c->analytic) return TUFRG_ERR_STATE;  // table-mode coarse-grid rows only
  return tufrg::set_refinement(c, s, kappa, lambda_on, (cudaStream_t)stream);
}

tufrg_status tufrg_atensor_bytes(const tufrg_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return TUFRG_ERR_ARG;
  size_t b = 0;
  const tufrg_status s = tufrg::atensor_bytes(c, &b);
  *bytes = (int64_t)b;
  return s;
}

tufrg_status tufrg_atensor_build(tufrg_ctx* c, void* stream) {
  if (!c || !c->d_V) return TUFRG_ERR_ARG;
  if (c->mesh) return TUFRG_ERR_STATE;  // the tensors of the coarse grid only
  return tufrg::atensor_build(c, (cudaStream_t)stream);
}

tufrg_status tufrg_project_atensor(tufrg_ctx* c, const double* y_dev, double* v_dev,
                                   void* stream) {
  if (!c || !y_dev || !v_dev || y_dev == v_dev) return TUFRG_ERR_ARG;
  return tufrg::atensor_project(c, y_dev, v_dev, (cudaStream_t)stream);
}

namespace {

// One right-hand side captured on the context's stream and instantiated.
tufrg_status capture_rhs(tufrg_ctx* c, const double* y_dev, double* dy_dev,
                         cudaGraphExec_t* exec) {
  cudaGraph_t g = nullptr;
  TUFRG_CUDA(cudaStreamBeginCapture(c->fstream, cudaStreamCaptureModeThreadLocal));
  const tufrg_status s = tufrg::rhs_device(c, c->p.precision, y_dev, dy_dev, false, c->fstream);
  cudaError_t e = cudaStreamEndCapture(c->fstream, &g);
  if (s != TUFRG_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  TUFRG_CUDA(e);
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) *exec = nullptr;
  TUFRG_CUDA(e);
  return TUFRG_OK;
}

// The right-hand side as a graph on the context's stream: one per (y, dy)
// pair, captured at the pair's first call and replayed after; the least
// recently used of the kRhsGraphs kept makes room for a new pair (an
// executable graph still in flight is freed when it completes).
tufrg_status rhs_graph(tufrg_ctx* c, const double* y_dev, double* dy_dev,
                       cudaGraphExec_t* exec) {
  tufrg_ctx::RhsGraph* slot = nullptr;
  for (auto& r : c->rhs_graphs)
    if (r.exec && r.y == y_dev && r.dy == dy_dev) {
      slot = &r;
      break;
    }
  if (!slot) {
    slot = &c->rhs_graphs[0];  // an empty entry, else the least recently used
    for (auto& r : c->rhs_graphs) {
      if (!r.exec) {
        slot = &r;
        break;
      }
      if (r.used < slot->used) slot = &r;
    }
    if (slot->exec) cudaGraphExecDestroy(slot->exec);
    *slot = tufrg_ctx::RhsGraph{};
    TUFRG_CHECK(capture_rhs(c, y_dev, dy_dev, &slot->exec));
    slot->y = y_dev;
    slot->dy = dy_dev;
  }
  slot->used = ++c->rhs_calls;
  *exec = slot->exec;
  return TUFRG_OK;
}

}  // namespace

tufrg_status tufrg_rhs(tufrg_ctx* c, double lambda, const double* y_dev, double* dy_dev,
                       void* stream) {
  if (!c || !y_dev || !dy_dev || y_dev == dy_dev || !finite_pos(lambda)) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!c->fstream) {
    TUFRG_CHECK(tufrg::launch_set_scalar(c->d_lambda, lambda, st));
    return tufrg::rhs_device(c, c->p.precision, y_dev, dy_dev, false, st);
  }
  TUFRG_CUDA(cudaEventRecord(c->ev_in, st));
  TUFRG_CUDA(cudaStreamWaitEvent(c->fstream, c->ev_in, 0));
  cudaGraphExec_t exec = nullptr;
  tufrg_status s = rhs_graph(c, y_dev, dy_dev, &exec);
  if (s == TUFRG_OK) s = tufrg::launch_set_scalar(c->d_lambda, lambda, c->fstream);
  if (s == TUFRG_OK) {
    const cudaError_t e = cudaGraphLaunch(exec, c->fstream);
    if (e != cudaSuccess) s = tufrg_cuda_fail_at(e, __FILE__, __LINE__);
  }
  if (cudaEventRecord(c->ev_out, c->fstream) != cudaSuccess ||
      cudaStreamWaitEvent(st, c->ev_out, 0) != cudaSuccess)
    return s == TUFRG_OK ? TUFRG_ERR_CUDA : s;
  return s;
}

tufrg_status tufrg_row_info(const tufrg_ctx* c, int32_t* nrow, int32_t* npair) {
  if (!c) return TUFRG_ERR_ARG;
  if (nrow) *nrow = c->nrow;
  if (npair) *npair = c->npair;
  return TUFRG_OK;
}

tufrg_status tufrg_shard_rows(tufrg_ctx* c, int32_t row_begin, int32_t row_end, void* stream) {
  if (!c || c->p.precision == TUFRG_FP64 || row_begin < 0 || row_end <= row_begin ||
      row_end > c->nrow)
    return TUFRG_ERR_ARG;
  if (c->mesh) return TUFRG_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  TUFRG_CUDA(cudaStreamSynchronize(st));
  c->shard_lo = row_begin;
  c->shard_hi = row_end;
  tufrg::flow_drop_graphs(c);
  double* lam[1] = {c->d_lambda};
  tufrg_ctx* self[1] = {c};
  return tufrg::view_build(c->view, self, 1, lam, nullptr, c->d_err, c->p.precision, 0, st);
}

tufrg_status tufrg_loop_rows(tufrg_ctx* c, double lambda, double* rows_dev, void* stream) {
  if (!c || !rows_dev || !finite_pos(lambda) || c->p.precision == TUFRG_FP64)
    return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  TUFRG_CHECK(tufrg::launch_set_scalar(c->d_lambda, lambda, st));
  TUFRG_CHECK(tufrg::launch_loops_tc_rows_multi(c->view, st));
  const size_t w = (size_t)(c->shard_hi - c->shard_lo) * c->npair;
  for (int ch = 0; ch < 2; ++ch) {
    const size_t o = ((size_t)ch * c->nrow + c->shard_lo) * c->npair;
    TUFRG_CUDA(cudaMemcpyAsync(rows_dev + o, c->view.d_rowres + o, sizeof(double) * w,
                               cudaMemcpyDeviceToDevice, st));
  }
  return TUFRG_OK;
}

tufrg_status tufrg_rhs_from_rows(tufrg_ctx* c, double lambda, const double* rows_dev,
                                 const double* y_dev, double* dy_dev, void* stream) {
  if (!c || !rows_dev || !y_dev || !dy_dev || y_dev == dy_dev || !finite_pos(lambda) ||
      !c->d_V)
    return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int arith = c->p.precision == TUFRG_FP64 ? TUFRG_FP64 : TUFRG_3XTF32;
  TUFRG_CHECK(tufrg::launch_set_scalar(c->d_lambda, lambda, st));
  TUFRG_CUDA(cudaMemcpyAsync(c->view.d_rowres, rows_dev,
                             sizeof(double) * 2 * (size_t)c->nrow * c->npair,
                             cudaMemcpyDeviceToDevice, st));
  const void* yin = y_dev;
  if (arith != TUFRG_FP64) {
    TUFRG_CHECK(tufrg::launch_to_f32(y_dev, c->d_y32, c->view.state_elems, st));
    yin = c->d_y32;
  }
  TUFRG_CHECK(tufrg::launch_project_multi(c->view, arith, yin, c->d_V, c->d_bt, c->d_fkey, st));
  return tufrg::launch_products_multi(c->view, arith, c->d_V, nullptr, dy_dev, false, st);
}

namespace {

tufrg_status check_opts(const tufrg_flow_opts* o) {
  if (!o) return TUFRG_ERR_ARG;
  if (!finite_pos(o->lambda0) || !finite_pos(o->lambda_min) || o->lambda_min >= o->lambda0)
    return TUFRG_ERR_ARG;
  if (!finite_pos(o->threshold) || !(o->rtol >= 0.0) || !(o->atol >= 0.0) ||
      o->rtol + o->atol <= 0.0 || !finite_pos(o->h0))
    return TUFRG_ERR_ARG;
  if (o->method != TUFRG_DOPRI5 && o->method != TUFRG_RK4) return TUFRG_ERR_ARG;
  if (o->n_checkpoints < 0 ||
      (o->n_checkpoints > 0 && (!o->checkpoints || !o->checkpoint_states_dev)))
    return TUFRG_ERR_ARG;
  for (int i = 0; i < o->n_checkpoints; ++i)
    if (!finite_pos(o->checkpoints[i])) return TUFRG_ERR_ARG;
  if (!(o->fp64_above >= 0.0) || !std::isfinite(o->fp64_above)) return TUFRG_ERR_ARG;
  return TUFRG_OK;
}

// flows run on the context's stream, ordered after / before the caller's
tufrg_status enter(tufrg_ctx* c, cudaStream_t user) {
  TUFRG_CUDA(cudaEventRecord(c->ev_in, user));
  TUFRG_CUDA(cudaStreamWaitEvent(c->fstream, c->ev_in, 0));
  return TUFRG_OK;
}

tufrg_status leave(tufrg_ctx* c, cudaStream_t user, tufrg_status s) {
  if (cudaEventRecord(c->ev_out, c->fstream) != cudaSuccess ||
      cudaStreamWaitEvent(user, c->ev_out, 0) != cudaSuccess)
    return s == TUFRG_OK ? TUFRG_ERR_CUDA : s;
  return s;
}

}  // namespace

tufrg_status tufrg_flow(tufrg_ctx* c, const tufrg_flow_opts* o, double* y_dev,
                        tufrg_result* res, void* stream) {
  if (!c || !y_dev || !res || o == nullptr || o->max_steps <= 0) return TUFRG_ERR_ARG;
  TUFRG_CHECK(check_opts(o));
  cudaStream_t user = (cudaStream_t)stream;
  TUFRG_CHECK(enter(c, user));
  tufrg_status s = tufrg::flow_init(c, o, y_dev, c->fstream);
  if (s == TUFRG_OK) s = tufrg::flow_step(c, o->max_steps, nullptr, c->fstream);
  tufrg_status s2 = tufrg::flow_state(c, y_dev, res, c->fstream);
  if (s == TUFRG_OK) s = s2;
  return leave(c, user, s);
}

tufrg_status tufrg_flow_init(tufrg_ctx* c, const tufrg_flow_opts* o, const double* y0_dev,
                             void* stream) {
  if (!c || !y0_dev) return TUFRG_ERR_ARG;
  TUFRG_CHECK(check_opts(o));
  cudaStream_t user = (cudaStream_t)stream;
  TUFRG_CHECK(enter(c, user));
  return leave(c, user, tufrg::flow_init(c, o, y0_dev, c->fstream));
}

tufrg_status tufrg_flow_step(tufrg_ctx* c, int32_t n_steps, tufrg_result* res, void* stream) {
  if (!c || n_steps < 0) return TUFRG_ERR_ARG;
  cudaStream_t user = (cudaStream_t)stream;
  TUFRG_CHECK(enter(c, user));
  return leave(c, user, tufrg::flow_step(c, n_steps, res, c->fstream));
}

tufrg_status tufrg_flow_state(tufrg_ctx* c, double* y_dev, tufrg_result* res, void* stream) {
  if (!c) return TUFRG_ERR_ARG;
  cudaStream_t user = (cudaStream_t)stream;
  TUFRG_CHECK(enter(c, user));
  return leave(c, user, tufrg::flow_state(c, y_dev, res, c->fstream));
}

tufrg_status tufrg_mu_for_density(double t, double tp, double n, int32_t nf_x, int32_t nf_y,
                                  double* mu_out) {
  if (!mu_out || nf_x < 2 || nf_y < 2 || !(n > 0.0 && n < 2.0) || !std::isfinite(t) ||
      !std::isfinite(tp))
    return TUFRG_ERR_ARG;
  std::vector<double> cx(nf_x), cy(nf_y);
  for (int i = 0; i < nf_x; ++i) cx[i] = std::cos(-M_PI + 2.0 * M_PI * i / nf_x);
  for (int i = 0; i < nf_y; ++i) cy[i] = std::cos(-M_PI + 2.0 * M_PI * i / nf_y);
  auto density = [&](double mu) {
    double below = 0.0;
    for (int i = 0; i < nf_x; ++i)
      for (int j = 0; j < nf_y; ++j) {
        double e0 = -2.0 * t * (cx[i] + cy[j]) - 4.0 * tp * cx[i] * cy[j];
        below += e0 < mu ? 1.0 : (e0 == mu ? 0.5 : 0.0);
      }
    return 2.0 * below / ((double)nf_x * nf_y);
  };
  double lo = -4.0 * std::fabs(t) - 4.0 * std::fabs(tp) - 1.0;
  double hi = 4.0 * std::fabs(t) + 4.0 * std::fabs(tp) + 1.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (density(mid) < n)
      lo = mid;
    else
      hi = mid;
  }
  *mu_out = 0.5 * (lo + hi);
  return TUFRG_OK;
}

tufrg_status tufrg_profile_loops(tufrg_ctx* c, double lambda, int32_t n, double* kernel_ms,
                                 double* stage_ms, void* stream) {
  if (!c || n < 1 || !finite_pos(lambda) || !kernel_ms || !stage_ms || !c->d_chi)
    return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  tufrg_status s = TUFRG_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) s = TUFRG_ERR_CUDA;
  double k = 0.0, g = 0.0;
  for (int i = 0; i < n && s == TUFRG_OK; ++i) {
    s = tufrg::launch_set_scalar(c->d_lambda, lambda, st);
    if (s == TUFRG_OK && cudaEventRecord(ev[2], st) != cudaSuccess) s = TUFRG_ERR_CUDA;
    if (s == TUFRG_OK && c->p.precision == TUFRG_FP64) {
      s = tufrg::launch_scale_tables(c, st);
      if (s == TUFRG_OK) s = tufrg::launch_loops_fp64_rows(c, st, ev);
    } else if (s == TUFRG_OK) {
      s = tufrg::launch_loops_tc_rows_multi(c->view, st, ev);
    }
    if (s == TUFRG_OK && cudaEventRecord(ev[3], st) != cudaSuccess) s = TUFRG_ERR_CUDA;
    float a = 0.f, b = 0.f;
    if (s == TUFRG_OK &&
        (cudaEventSynchronize(ev[3]) != cudaSuccess ||
         cudaEventElapsedTime(&a, ev[0], ev[1]) != cudaSuccess ||
         cudaEventElapsedTime(&b, ev[2], ev[3]) != cudaSuccess))
      s = TUFRG_ERR_CUDA;
    k += a;
    g += b;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  TUFRG_CHECK(s);
  *kernel_ms = k / n;
  *stage_ms = g / n;
  return tufrg_check(c, stream);
}

tufrg_status tufrg_check(tufrg_ctx* c, void* stream) {
  if (!c) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int err = 0;
  TUFRG_CUDA(cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TUFRG_CUDA(cudaStreamSynchronize(st));
  if (err) {
    TUFRG_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    TUFRG_CUDA(cudaStreamSynchronize(st));
    return TUFRG_ERR_TIMEOUT;
  }
  return TUFRG_OK;
}

const char* tufrg_last_cuda_error(void) {
  if (g_last_cuda_error == cudaSuccess) return "";
  return g_last_cuda_where[0] ? g_last_cuda_where : cudaGetErrorName(g_last_cuda_error);
}

const char* tufrg_status_string(tufrg_status s) {
  switch (s) {
    case TUFRG_OK: return "ok";
    case TUFRG_ERR_ARG: return "invalid argument";
    case TUFRG_ERR_CUDA: return "CUDA error";
    case TUFRG_ERR_NONFINITE: return "non-finite state";
    case TUFRG_ERR_STEP_UNDERFLOW: return "step size underflow";
    case TUFRG_ERR_TIMEOUT: return "device wait timed out";
    case TUFRG_ERR_OOM: return "out of device memory";
    case TUFRG_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

}  // extern "C"
