"""ctypes binding of include/tufrg.h (argument marshalling only).

Every function has the C name and takes plain numbers and pointers; device
pointers are passed as integers (e.g. torch.Tensor.data_ptr()), streams as
the integer value of a cudaStream_t.  A non-zero status raises TufrgError.
The library must have been built (paper_1604_06296_gb300.build); there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, byref, c_double, c_int32, c_int64, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtufrg.so")

TUFRG_FP64, TUFRG_3XTF32, TUFRG_BF16X3 = 0, 1, 2
TUFRG_DOPRI5, TUFRG_RK4 = 0, 1
STATUS = {0: "TUFRG_OK", -1: "TUFRG_ERR_ARG", -2: "TUFRG_ERR_CUDA", -3: "TUFRG_ERR_NONFINITE",
          -4: "TUFRG_ERR_STEP_UNDERFLOW", -5: "TUFRG_ERR_TIMEOUT", -6: "TUFRG_ERR_OOM",
          -7: "TUFRG_ERR_STATE"}


class TufrgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class tufrg_params(Structure):
    _fields_ = [("lattice", c_int32), ("t", c_double), ("tp", c_double), ("mu", c_double),
                ("U", c_double), ("n_bonds", c_int32), ("bonds", POINTER(c_int32)),
                ("nc_x", c_int32), ("nc_y", c_int32), ("nf_x", c_int32), ("nf_y", c_int32),
                ("precision", c_int32), ("feedback", c_int32)]


class tufrg_flow_opts(Structure):
    _fields_ = [("lambda0", c_double), ("lambda_min", c_double), ("threshold", c_double),
                ("rtol", c_double), ("atol", c_double), ("h0", c_double),
                ("method", c_int32), ("max_steps", c_int32), ("n_checkpoints", c_int32),
                ("checkpoints", POINTER(c_double)), ("checkpoint_states_dev", c_void_p),
                ("fp64_above", c_double)]


class tufrg_result(Structure):
    _fields_ = [("lambda_c", c_double), ("h_next", c_double), ("diverged", c_int32),
                ("finished", c_int32), ("channel", c_int32), ("l_index", c_int32),
                ("m", c_int32), ("n", c_int32), ("max_abs", c_double),
                ("lambda_switch", c_double),
                ("n_rhs", c_int64), ("n_accepted", c_int64), ("n_rejected", c_int64),
                ("lambda_surrogate_off", c_double), ("n_rhs_surrogate", c_int64),
                ("n_judges", c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class tufrg_tune_report(Structure):
    _fields_ = [("n_candidates", c_int32), ("kbps", c_int32 * 16), ("ms", c_double * 16),
                ("chosen", c_int32), ("kbps_default", c_int32)]

    def as_dict(self):
        n = self.n_candidates
        return {"kbps": list(self.kbps[:n]), "ms": list(self.ms[:n]),
                "chosen": self.kbps[self.chosen], "kbps_default": self.kbps_default}


_lib = None

# name -> (argtypes, restype); restype c_int32 means a tufrg_status to check
SIGNATURES = {
    "tufrg_setup": ([POINTER(tufrg_params), c_void_p, POINTER(c_void_p)], c_int32),
    "tufrg_setup_mesh": ([POINTER(tufrg_params), c_int32, c_int32, POINTER(c_int32),
                          POINTER(c_double), POINTER(c_double), c_void_p, POINTER(c_void_p)],
                         c_int32),
    "tufrg_destroy": ([c_void_p], None),
    "tufrg_dims": ([c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)], c_int32),
    "tufrg_eval_formfactors": ([c_int32, POINTER(c_int32), c_int32, POINTER(c_double),
                                POINTER(c_double), POINTER(c_double), POINTER(c_int32)],
                               c_int32),
    "tufrg_loops": ([c_void_p, c_double, c_void_p, c_void_p], c_int32),
    "tufrg_row_info": ([c_void_p, POINTER(c_int32), POINTER(c_int32)], c_int32),
    "tufrg_shard_rows": ([c_void_p, c_int32, c_int32, c_void_p], c_int32),
    "tufrg_loop_rows": ([c_void_p, c_double, c_void_p, c_void_p], c_int32),
    "tufrg_rhs_from_rows": ([c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_void_p],
                            c_int32),
    "tufrg_project": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "tufrg_products": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "tufrg_rhs": ([c_void_p, c_double, c_void_p, c_void_p, c_void_p], c_int32),
    "tufrg_flow": ([c_void_p, POINTER(tufrg_flow_opts), c_void_p, POINTER(tufrg_result),
                    c_void_p], c_int32),
    "tufrg_flow_init": ([c_void_p, POINTER(tufrg_flow_opts), c_void_p, c_void_p], c_int32),
    "tufrg_flow_step": ([c_void_p, c_int32, POINTER(tufrg_result), c_void_p], c_int32),
    "tufrg_flow_state": ([c_void_p, c_void_p, POINTER(tufrg_result), c_void_p], c_int32),
    "tufrg_loops_noalloc": ([POINTER(tufrg_params), c_double, c_void_p, c_void_p], c_int32),
    "tufrg_mu_for_density": ([c_double, c_double, c_double, c_int32, c_int32,
                              POINTER(c_double)], c_int32),
    "tufrg_check": ([c_void_p, c_void_p], c_int32),
    "tufrg_selftest_wait": ([c_void_p, c_int32, c_void_p], c_int32),
    "tufrg_selftest_convert": ([c_void_p, c_void_p, c_void_p, c_int64, c_void_p], c_int32),
    "tufrg_atensor_bytes": ([c_void_p, POINTER(c_int64)], c_int32),
    "tufrg_set_refinement": ([c_void_p, c_int32, c_double, c_double, c_void_p], c_int32),
    "tufrg_atensor_build": ([c_void_p, c_void_p], c_int32),
    "tufrg_project_atensor": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "tufrg_autotune": ([c_void_p, c_double, POINTER(tufrg_tune_report), c_void_p], c_int32),
    "tufrg_batch_setup": ([c_int32, POINTER(tufrg_params), c_void_p, POINTER(c_void_p)],
                          c_int32),
    "tufrg_batch_destroy": ([c_void_p], None),
    "tufrg_batch_dims": ([c_void_p, c_int32, POINTER(c_int32), POINTER(c_int32),
                          POINTER(c_int64), POINTER(c_int64)], c_int32),
    "tufrg_batch_loops": ([c_void_p, POINTER(c_double), c_void_p, c_void_p], c_int32),
    "tufrg_batch_rhs": ([c_void_p, POINTER(c_double), c_void_p, c_void_p, c_void_p], c_int32),
    "tufrg_batch_flow": ([c_void_p, POINTER(tufrg_flow_opts), c_void_p, POINTER(tufrg_result),
                          POINTER(c_int32), c_void_p], c_int32),
    "tufrg_batch_autotune": ([c_void_p, c_double, POINTER(tufrg_tune_report), c_void_p],
                             c_int32),
    "tufrg_batch_check": ([c_void_p, c_void_p], c_int32),
    "tufrg_surrogate_create": ([c_int32, c_int32, c_int32, ctypes.c_uint64, POINTER(c_void_p)],
                               c_int32),
    "tufrg_surrogate_destroy": ([c_void_p], None),
    "tufrg_surrogate_n_params": ([c_void_p, POINTER(c_int64)], c_int32),
    "tufrg_surrogate_get_params": ([c_void_p, POINTER(ctypes.c_float), c_void_p], c_int32),
    "tufrg_surrogate_set_params": ([c_void_p, POINTER(ctypes.c_float), c_void_p], c_int32),
    "tufrg_surrogate_get_scaling": ([c_void_p, POINTER(ctypes.c_float), POINTER(ctypes.c_float),
                                     c_void_p], c_int32),
    "tufrg_surrogate_set_scaling": ([c_void_p, POINTER(ctypes.c_float), POINTER(ctypes.c_float),
                                     c_void_p], c_int32),
    "tufrg_surrogate_samples": ([c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p],
                                c_int32),
    "tufrg_surrogate_predict": ([c_void_p, c_void_p, c_int64, c_void_p, c_void_p], c_int32),
    "tufrg_surrogate_loss_grad": ([c_void_p, c_void_p, c_void_p, c_int64, POINTER(c_double),
                                   POINTER(ctypes.c_float), c_void_p], c_int32),
    "tufrg_surrogate_train": ([c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_double,
                               ctypes.c_uint64, POINTER(c_double), c_void_p], c_int32),
    "tufrg_surrogate_attach": ([c_void_p, c_void_p, c_int32, c_double], c_int32),
    "tufrg_profile_loops": ([c_void_p, c_double, c_int32, POINTER(c_double), POINTER(c_double),
                             c_void_p], c_int32),
    "tufrg_batch_profile_loops": ([c_void_p, c_double, c_int32, POINTER(c_double),
                                   POINTER(c_double), c_void_p], c_int32),
    "tufrg_status_string": ([c_int32], ctypes.c_char_p),
    "tufrg_last_cuda_error": ([], ctypes.c_char_p),
}


def lib():
    """The loaded libtufrg.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_1604_06296_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != 0:
        detail = lib().tufrg_last_cuda_error().decode() if status in (-2, -6) else ""
        raise TufrgError(status, f"{where} ({detail})" if detail else where)


def _dptr(p) -> c_void_p:
    return c_void_p(int(p) if p else 0)


def tufrg_setup(params: tufrg_params, stream: int = 0) -> c_void_p:
    ctx = c_void_p()
    _check(lib().tufrg_setup(byref(params), _dptr(stream), byref(ctx)), "tufrg_setup")
    return ctx


def tufrg_setup_mesh(params: tufrg_params, m: int, points, w_p, w_cd,
                     stream: int = 0) -> c_void_p:
    """points: int32 [n][2] lattice coordinates; w_p, w_cd: float64 [n] (host)."""
    pts = np.ascontiguousarray(points, dtype=np.int32).reshape(-1, 2)
    wp = np.ascontiguousarray(w_p, dtype=np.float64).reshape(-1)
    wc = np.ascontiguousarray(w_cd, dtype=np.float64).reshape(-1)
    if len(wp) != len(pts) or len(wc) != len(pts):
        raise ValueError("points, w_p and w_cd must have the same length")
    ctx = c_void_p()
    _check(lib().tufrg_setup_mesh(byref(params), int(m), len(pts),
                                  pts.ctypes.data_as(POINTER(c_int32)),
                                  wp.ctypes.data_as(POINTER(c_double)),
                                  wc.ctypes.data_as(POINTER(c_double)), _dptr(stream),
                                  byref(ctx)), "tufrg_setup_mesh")
    return ctx


def tufrg_destroy(ctx: c_void_p) -> None:
    lib().tufrg_destroy(ctx)


def tufrg_dims(ctx: c_void_p) -> tuple[int, int, int]:
    nl, nff, nb = c_int32(), c_int32(), c_int32()
    _check(lib().tufrg_dims(ctx, byref(nl), byref(nff), byref(nb)), "tufrg_dims")
    return nl.value, nff.value, nb.value


def tufrg_eval_formfactors(bonds, kx, ky):
    """bonds: int32 array [n][2]; kx, ky: float64 arrays [n]. Returns [Nff][n]."""
    b = np.ascontiguousarray(bonds, dtype=np.int32)
    kx = np.ascontiguousarray(kx, dtype=np.float64)
    ky = np.ascontiguousarray(ky, dtype=np.float64)
    nff = c_int32()
    bp = b.ctypes.data_as(POINTER(c_int32))
    _check(lib().tufrg_eval_formfactors(len(b), bp, 0, None, None, None, byref(nff)),
           "tufrg_eval_formfactors")
    out = np.empty((nff.value, len(kx)), dtype=np.float64)
    _check(lib().tufrg_eval_formfactors(len(b), bp, len(kx), kx.ctypes.data_as(POINTER(c_double)),
                                        ky.ctypes.data_as(POINTER(c_double)),
                                        out.ctypes.data_as(POINTER(c_double)), None),
           "tufrg_eval_formfactors")
    return out


def tufrg_loops(ctx, lam: float, chi_dot_dev: int, stream: int = 0) -> None:
    _check(lib().tufrg_loops(ctx, lam, _dptr(chi_dot_dev), _dptr(stream)), "tufrg_loops")


def tufrg_project(ctx, y_dev: int, v_dev: int, stream: int = 0) -> None:
    _check(lib().tufrg_project(ctx, _dptr(y_dev), _dptr(v_dev), _dptr(stream)), "tufrg_project")


def tufrg_products(ctx, v_dev: int, chi_dev: int, dy_dev: int, stream: int = 0) -> None:
    _check(lib().tufrg_products(ctx, _dptr(v_dev), _dptr(chi_dev), _dptr(dy_dev),
                                _dptr(stream)), "tufrg_products")


def tufrg_rhs(ctx, lam: float, y_dev: int, dy_dev: int, stream: int = 0) -> None:
    _check(lib().tufrg_rhs(ctx, lam, _dptr(y_dev), _dptr(dy_dev), _dptr(stream)), "tufrg_rhs")


def tufrg_flow(ctx, opts: tufrg_flow_opts, y_dev: int, stream: int = 0) -> tufrg_result:
    res = tufrg_result()
    _check(lib().tufrg_flow(ctx, byref(opts), _dptr(y_dev), byref(res), _dptr(stream)),
           "tufrg_flow")
    return res


def tufrg_flow_init(ctx, opts: tufrg_flow_opts, y0_dev: int, stream: int = 0) -> None:
    _check(lib().tufrg_flow_init(ctx, byref(opts), _dptr(y0_dev), _dptr(stream)),
           "tufrg_flow_init")


def tufrg_flow_step(ctx, n_steps: int, stream: int = 0) -> tufrg_result:
    res = tufrg_result()
    _check(lib().tufrg_flow_step(ctx, n_steps, byref(res), _dptr(stream)), "tufrg_flow_step")
    return res


def tufrg_flow_state(ctx, y_dev: int, stream: int = 0) -> tufrg_result:
    res = tufrg_result()
    _check(lib().tufrg_flow_state(ctx, _dptr(y_dev), byref(res), _dptr(stream)),
           "tufrg_flow_state")
    return res


def tufrg_row_info(ctx) -> tuple[int, int]:
    """(nrow, npair): loop rows and parity-allowed pairs of the context."""
    nrow, npair = c_int32(), c_int32()
    _check(lib().tufrg_row_info(ctx, byref(nrow), byref(npair)), "tufrg_row_info")
    return nrow.value, npair.value


def tufrg_shard_rows(ctx, row_begin: int, row_end: int, stream: int = 0) -> None:
    _check(lib().tufrg_shard_rows(ctx, row_begin, row_end, _dptr(stream)), "tufrg_shard_rows")


def tufrg_loop_rows(ctx, lam: float, rows_dev: int, stream: int = 0) -> None:
    _check(lib().tufrg_loop_rows(ctx, lam, _dptr(rows_dev), _dptr(stream)), "tufrg_loop_rows")


def tufrg_rhs_from_rows(ctx, lam: float, rows_dev: int, y_dev: int, dy_dev: int,
                        stream: int = 0) -> None:
    _check(lib().tufrg_rhs_from_rows(ctx, lam, _dptr(rows_dev), _dptr(y_dev), _dptr(dy_dev),
                                     _dptr(stream)), "tufrg_rhs_from_rows")


def tufrg_loops_noalloc(params: tufrg_params, lam: float, chi_dot_dev: int,
                        stream: int = 0) -> None:
    """Loops without any device allocation (see include/tufrg.h)."""
    _check(lib().tufrg_loops_noalloc(byref(params), lam, _dptr(chi_dot_dev), _dptr(stream)),
           "tufrg_loops_noalloc")


def tufrg_mu_for_density(t: float, tp: float, n: float, nf_x: int, nf_y: int) -> float:
    mu = c_double()
    _check(lib().tufrg_mu_for_density(t, tp, n, nf_x, nf_y, byref(mu)), "tufrg_mu_for_density")
    return mu.value


def tufrg_check(ctx, stream: int = 0) -> None:
    _check(lib().tufrg_check(ctx, _dptr(stream)), "tufrg_check")


def tufrg_selftest_wait(ctx, wait_us: int, stream: int = 0) -> None:
    _check(lib().tufrg_selftest_wait(ctx, int(wait_us), _dptr(stream)), "tufrg_selftest_wait")


def tufrg_selftest_convert(x_ptr: int, y32_ptr: int, back_ptr: int, n: int,
                           stream: int = 0) -> None:
    _check(lib().tufrg_selftest_convert(_dptr(x_ptr), _dptr(y32_ptr), _dptr(back_ptr), int(n),
                                        _dptr(stream)), "tufrg_selftest_convert")


def tufrg_set_refinement(ctx, s: int, kappa: float, lambda_on: float, stream: int = 0) -> None:
    _check(lib().tufrg_set_refinement(ctx, int(s), float(kappa), float(lambda_on), _dptr(stream)),
           "tufrg_set_refinement")


def tufrg_atensor_bytes(ctx) -> int:
    b = c_int64()
    _check(lib().tufrg_atensor_bytes(ctx, byref(b)), "tufrg_atensor_bytes")
    return b.value


def tufrg_atensor_build(ctx, stream: int = 0) -> None:
    _check(lib().tufrg_atensor_build(ctx, _dptr(stream)), "tufrg_atensor_build")


def tufrg_project_atensor(ctx, y_ptr: int, v_ptr: int, stream: int = 0) -> None:
    _check(lib().tufrg_project_atensor(ctx, _dptr(y_ptr), _dptr(v_ptr), _dptr(stream)),
           "tufrg_project_atensor")


def tufrg_status_string(status: int) -> str:
    return lib().tufrg_status_string(status).decode()


def tufrg_autotune(ctx, lam: float, stream: int = 0) -> tufrg_tune_report:
    rep = tufrg_tune_report()
    _check(lib().tufrg_autotune(ctx, lam, byref(rep), _dptr(stream)), "tufrg_autotune")
    return rep


def tufrg_batch_setup(params, stream: int = 0) -> c_void_p:
    """params: a ctypes array of tufrg_params."""
    b = c_void_p()
    _check(lib().tufrg_batch_setup(len(params), params, _dptr(stream), byref(b)),
           "tufrg_batch_setup")
    return b


def tufrg_batch_destroy(b) -> None:
    lib().tufrg_batch_destroy(b)


def tufrg_batch_dims(b, point: int) -> tuple[int, int, int, int]:
    nl, nff, so, lo = c_int32(), c_int32(), c_int64(), c_int64()
    _check(lib().tufrg_batch_dims(b, point, byref(nl), byref(nff), byref(so), byref(lo)),
           "tufrg_batch_dims")
    return nl.value, nff.value, so.value, lo.value


def _doubles(x):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a, a.ctypes.data_as(POINTER(c_double))


def tufrg_batch_loops(b, lam, chi_dev: int, stream: int = 0) -> None:
    a, ptr = _doubles(lam)
    _check(lib().tufrg_batch_loops(b, ptr, _dptr(chi_dev), _dptr(stream)), "tufrg_batch_loops")


def tufrg_batch_rhs(b, lam, y_dev: int, dy_dev: int, stream: int = 0) -> None:
    a, ptr = _doubles(lam)
    _check(lib().tufrg_batch_rhs(b, ptr, _dptr(y_dev), _dptr(dy_dev), _dptr(stream)),
           "tufrg_batch_rhs")


def tufrg_batch_flow(b, n_points: int, opts: tufrg_flow_opts, y_dev: int, stream: int = 0):
    """Returns (status, results, per-point statuses); a failing point does not raise."""
    res = (tufrg_result * n_points)()
    st = (c_int32 * n_points)()
    s = lib().tufrg_batch_flow(b, byref(opts), _dptr(y_dev), res, st, _dptr(stream))
    if s not in (0, -3, -4):
        _check(s, "tufrg_batch_flow")
    return s, list(res), list(st)


def tufrg_batch_autotune(b, lam: float, stream: int = 0) -> tufrg_tune_report:
    rep = tufrg_tune_report()
    _check(lib().tufrg_batch_autotune(b, lam, byref(rep), _dptr(stream)), "tufrg_batch_autotune")
    return rep


def tufrg_batch_check(b, stream: int = 0) -> None:
    _check(lib().tufrg_batch_check(b, _dptr(stream)), "tufrg_batch_check")


def tufrg_surrogate_create(n_out: int, width: int, depth: int, seed: int) -> c_void_p:
    s = c_void_p()
    _check(lib().tufrg_surrogate_create(n_out, width, depth, seed, byref(s)),
           "tufrg_surrogate_create")
    return s


def tufrg_surrogate_destroy(s) -> None:
    lib().tufrg_surrogate_destroy(s)


def tufrg_surrogate_n_params(s) -> int:
    n = c_int64()
    _check(lib().tufrg_surrogate_n_params(s, byref(n)), "tufrg_surrogate_n_params")
    return n.value


def tufrg_surrogate_get_params(s, stream: int = 0):
    out = np.empty(tufrg_surrogate_n_params(s), dtype=np.float32)
    _check(lib().tufrg_surrogate_get_params(s, out.ctypes.data_as(POINTER(ctypes.c_float)),
                                            _dptr(stream)), "tufrg_surrogate_get_params")
    return out


def tufrg_surrogate_set_params(s, params, stream: int = 0) -> None:
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().tufrg_surrogate_set_params(s, a.ctypes.data_as(POINTER(ctypes.c_float)),
                                            _dptr(stream)), "tufrg_surrogate_set_params")


def tufrg_surrogate_samples(ctx, s, lam: float, x_dev: int, t_dev: int, stream: int = 0) -> None:
    _check(lib().tufrg_surrogate_samples(ctx, s, lam, _dptr(x_dev), _dptr(t_dev), _dptr(stream)),
           "tufrg_surrogate_samples")


def tufrg_surrogate_predict(s, x_dev: int, n: int, y_dev: int, stream: int = 0) -> None:
    _check(lib().tufrg_surrogate_predict(s, _dptr(x_dev), n, _dptr(y_dev), _dptr(stream)),
           "tufrg_surrogate_predict")


def tufrg_surrogate_loss_grad(s, x_dev: int, t_dev: int, n: int, stream: int = 0):
    loss = c_double()
    g = np.empty(tufrg_surrogate_n_params(s), dtype=np.float32)
    _check(lib().tufrg_surrogate_loss_grad(s, _dptr(x_dev), _dptr(t_dev), n, byref(loss),
                                           g.ctypes.data_as(POINTER(ctypes.c_float)),
                                           _dptr(stream)), "tufrg_surrogate_loss_grad")
    return loss.value, g


def tufrg_surrogate_train(s, x_dev: int, t_dev: int, n: int, epochs: int, batch: int, lr: float,
                          seed: int, stream: int = 0):
    hist = (c_double * epochs)()
    _check(lib().tufrg_surrogate_train(s, _dptr(x_dev), _dptr(t_dev), n, epochs, batch, lr, seed,
                                       hist, _dptr(stream)), "tufrg_surrogate_train")
    return list(hist)


def tufrg_surrogate_attach(ctx, s, judge_every: int = 8, tol: float = 1e-3) -> None:
    _check(lib().tufrg_surrogate_attach(ctx, s, judge_every, tol), "tufrg_surrogate_attach")


def tufrg_surrogate_get_scaling(s, n_out: int, stream: int = 0):
    sh = np.empty(n_out, dtype=np.float32)
    sc = np.empty(n_out, dtype=np.float32)
    _check(lib().tufrg_surrogate_get_scaling(s, sh.ctypes.data_as(POINTER(ctypes.c_float)),
                                             sc.ctypes.data_as(POINTER(ctypes.c_float)),
                                             _dptr(stream)), "tufrg_surrogate_get_scaling")
    return sh, sc


def tufrg_surrogate_set_scaling(s, shift, scale, stream: int = 0) -> None:
    if shift is None:
        _check(lib().tufrg_surrogate_set_scaling(s, None, None, _dptr(stream)),
               "tufrg_surrogate_set_scaling")
        return
    a = np.ascontiguousarray(shift, dtype=np.float32)
    b = np.ascontiguousarray(scale, dtype=np.float32)
    _check(lib().tufrg_surrogate_set_scaling(s, a.ctypes.data_as(POINTER(ctypes.c_float)),
                                             b.ctypes.data_as(POINTER(ctypes.c_float)),
                                             _dptr(stream)), "tufrg_surrogate_set_scaling")


def tufrg_profile_loops(ctx, lam: float, n: int, stream: int = 0):
    """(kernel ms, stage ms) averaged over n loop contractions."""
    k, g = c_double(), c_double()
    _check(lib().tufrg_profile_loops(ctx, lam, n, byref(k), byref(g), _dptr(stream)),
           "tufrg_profile_loops")
    return k.value, g.value


def tufrg_batch_profile_loops(b, lam: float, n: int, stream: int = 0):
    k, g = c_double(), c_double()
    _check(lib().tufrg_batch_profile_loops(b, lam, n, byref(k), byref(g), _dptr(stream)),
           "tufrg_batch_profile_loops")
    return k.value, g.value
