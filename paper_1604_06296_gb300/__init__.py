"""GB300-native TUfRG Lambda-flow right-hand side (arXiv:1604.06296).

The computation lives in libtufrg.so (CUDA for sm_103a behind the C ABI of
include/tufrg.h).  ``_abi`` is the thin ctypes binding with the C names;
``Solver`` marshals torch tensors (device memory and the current stream) to
it.  There is no CPU or PyTorch fallback: a missing or unloadable library
raises.
"""
from __future__ import annotations

import numpy as np

from . import _abi
from ._abi import (TUFRG_3XTF32, TUFRG_BF16X3, TUFRG_DOPRI5, TUFRG_FP64, TUFRG_RK4,  # noqa: F401
                   TufrgError, tufrg_destroy, tufrg_dims, tufrg_eval_formfactors,
                   tufrg_flow, tufrg_flow_init, tufrg_flow_state, tufrg_flow_step,
                   tufrg_loops, tufrg_mu_for_density, tufrg_products, tufrg_project,
                   tufrg_rhs, tufrg_setup, tufrg_status_string)

PRECISIONS = {"fp64": TUFRG_FP64, "3xtf32": TUFRG_3XTF32, "bf16x3": TUFRG_BF16X3}
CHANNEL_KIND = {0: "pairing", 1: "magnetic", 2: "charge"}


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Solver:
    """One phase-diagram point on the current CUDA device.

    Arrays are float64 CUDA tensors: state y = (P, C, D) [3][Nl][Nff][Nff],
    loops [2][Nl][Nff][Nff], projected couplings [3][Nl][Nff][Nff].
    """

    def __init__(self, t, tp, mu, U, bonds, nc, nf, precision="fp64", feedback=True,
                 ncy=None, nfy=None, mesh=None):
        """mesh: None (the coarse grid) or (m, points [n][2], w_p [n], w_cd [n]),
        a non-uniform mesh of lattice points l = -pi + 2 pi j / (nc m) with the
        quadrature weights of mesh_P and mesh_CD (Sec. 4)."""
        self._bonds = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p = _abi.tufrg_params()
        p.lattice = 0
        p.t, p.tp, p.mu, p.U = float(t), float(tp), float(mu), float(U)
        p.n_bonds = len(self._bonds)
        p.bonds = self._bonds.ctypes.data_as(_abi.POINTER(_abi.c_int32))
        p.nc_x, p.nc_y = int(nc), int(ncy or nc)
        p.nf_x, p.nf_y = int(nf), int(nfy or nf)
        p.precision = prec
        p.feedback = 1 if feedback else 0
        self.params = p
        if mesh is None:
            self.ctx = tufrg_setup(p, _stream())
        else:
            m, points, w_p, w_cd = mesh
            self.ctx = _abi.tufrg_setup_mesh(p, int(m), points, w_p, w_cd, _stream())
        self.nl, self.nff, self.nb = tufrg_dims(self.ctx)

    # -- helpers -------------------------------------------------------------
    def _check(self, x, lead):
        import torch
        shape = (lead, self.nl, self.nff, self.nff)
        if (not isinstance(x, torch.Tensor) or x.dtype != torch.float64 or not x.is_cuda
                or not x.is_contiguous() or tuple(x.shape) != shape):
            raise ValueError(f"expected a contiguous float64 CUDA tensor of shape {shape}")
        return x.data_ptr()

    def empty(self, lead=3):
        import torch
        return torch.empty((lead, self.nl, self.nff, self.nff), dtype=torch.float64,
                           device="cuda")

    def zeros(self, lead=3):
        return self.empty(lead).zero_()

    # -- steps of the right-hand side ---------------------------------------
    def loops(self, lam, out=None):
        out = self.empty(2) if out is None else out
        tufrg_loops(self.ctx, float(lam), self._check(out, 2), _stream())
        return out

    def project(self, y, out=None):
        out = self.empty(3) if out is None else out
        tufrg_project(self.ctx, self._check(y, 3), self._check(out, 3), _stream())
        return out

    def set_refinement(self, s=5, kappa=8.0, lambda_on=float("inf")):
        """Fermi-surface refinement of the loop cells (s = 1: off)."""
        lam_on = 1e300 if lambda_on == float("inf") else float(lambda_on)
        _abi.tufrg_set_refinement(self.ctx, int(s), float(kappa), lam_on, _stream())

    def atensor_bytes(self):
        """Device bytes of the precomputed projection tensors (App. C)."""
        return _abi.tufrg_atensor_bytes(self.ctx)

    def atensor_build(self):
        _abi.tufrg_atensor_build(self.ctx, _stream())

    def project_atensor(self, y, out=None):
        """Step i from the precomputed tensors (after atensor_build)."""
        out = self.empty(3) if out is None else out
        _abi.tufrg_project_atensor(self.ctx, self._check(y, 3), self._check(out, 3), _stream())
        return out

    def products(self, v, chi, out=None):
        out = self.empty(3) if out is None else out
        tufrg_products(self.ctx, self._check(v, 3), self._check(chi, 2), self._check(out, 3),
                       _stream())
        return out

    def rhs(self, lam, y, out=None):
        out = self.empty(3) if out is None else out
        tufrg_rhs(self.ctx, float(lam), self._check(y, 3), self._check(out, 3), _stream())
        return out

    def _opts(self, lambda0, lambda_min, threshold, rtol, atol, h0, method, max_steps,
              checkpoints, fp64_above=0.0):
        import torch
        o = _abi.tufrg_flow_opts()
        o.lambda0, o.lambda_min, o.threshold = float(lambda0), float(lambda_min), float(threshold)
        o.rtol, o.atol, o.h0 = float(rtol), float(atol), float(h0)
        o.method = TUFRG_RK4 if method == "rk4" else TUFRG_DOPRI5
        o.max_steps = int(max_steps)
        o.fp64_above = float(fp64_above)
        cks = np.ascontiguousarray(np.asarray(checkpoints, dtype=np.float64))
        states = torch.zeros((len(cks), 3, self.nl, self.nff, self.nff), dtype=torch.float64,
                             device="cuda")
        o.n_checkpoints = len(cks)
        o.checkpoints = cks.ctypes.data_as(_abi.POINTER(_abi.c_double)) if len(cks) else None
        o.checkpoint_states_dev = states.data_ptr() if len(cks) else None
        self._keep = (cks, states)   # alive while the flow may write checkpoints
        return o, states

    @staticmethod
    def _result(r):
        d = r.as_dict()
        d["diverged"], d["finished"] = bool(d["diverged"]), bool(d["finished"])
        d["kind"] = CHANNEL_KIND.get(d["channel"])
        return d

    def flow(self, y=None, lambda0=10.0, lambda_min=1e-3, threshold=50.0, rtol=1e-8,
             atol=1e-10, h0=0.05, method="dopri5", max_steps=100000, checkpoints=(),
             fp64_above=0.0):
        """Integrates the flow in place of y (zeros = bare U start).

        Returns (y, result dict, checkpoint states [n][3][Nl][Nff][Nff])."""
        y = self.zeros(3) if y is None else y
        o, states = self._opts(lambda0, lambda_min, threshold, rtol, atol, h0, method,
                               max_steps, checkpoints, fp64_above)
        r = tufrg_flow(self.ctx, o, self._check(y, 3), _stream())
        return y, self._result(r), states

    def flow_init(self, y0=None, lambda0=10.0, lambda_min=1e-3, threshold=50.0, rtol=1e-8,
                  atol=1e-10, h0=0.05, method="dopri5", checkpoints=(), fp64_above=0.0):
        """Starts a stepwise flow; returns the checkpoint-state tensor."""
        y0 = self.zeros(3) if y0 is None else y0
        o, states = self._opts(lambda0, lambda_min, threshold, rtol, atol, h0, method, 1,
                               checkpoints, fp64_above)
        tufrg_flow_init(self.ctx, o, self._check(y0, 3), _stream())
        return states

    def flow_step(self, n_steps=1):
        return self._result(tufrg_flow_step(self.ctx, int(n_steps), _stream()))

    def flow_state(self, out=None):
        out = self.empty(3) if out is None else out
        r = tufrg_flow_state(self.ctx, self._check(out, 3), _stream())
        return out, self._result(r)

    def attach_surrogate(self, surrogate, judge_every=8, tol=1e-3):
        """Flows use the surrogate's loops while the exact judge accepts them."""
        _abi.tufrg_surrogate_attach(self.ctx, surrogate.s if surrogate else None,
                                    int(judge_every), float(tol))

    def profile_loops(self, lam=0.5, n=5):
        """(contraction kernel ms, loop stage ms), CUDA events inside the library."""
        return _abi.tufrg_profile_loops(self.ctx, float(lam), int(n), _stream())

    def autotune(self, lam=1.0):
        """Tile autotuning of the tensor-core loops; returns the timing report."""
        return _abi.tufrg_autotune(self.ctx, float(lam), _stream()).as_dict()

    def check(self):
        """Raise TufrgError if a device wait gave up since the last check."""
        _abi.tufrg_check(self.ctx, _stream())

    def selftest_wait(self, wait_us=20000):
        """Launch one bounded wait that nothing completes (diagnostic)."""
        _abi.tufrg_selftest_wait(self.ctx, int(wait_us), _stream())

    def close(self):
        if getattr(self, "ctx", None) is not None:
            tufrg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_params(t, tp, mu, U, bonds, nc, nf, precision="bf16x3", feedback=True, ncy=None,
                nfy=None):
    """A tufrg_params and the bond array it points to (keep both alive)."""
    b = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
    p = _abi.tufrg_params()
    p.lattice = 0
    p.t, p.tp, p.mu, p.U = float(t), float(tp), float(mu), float(U)
    p.n_bonds = len(b)
    p.bonds = b.ctypes.data_as(_abi.POINTER(_abi.c_int32))
    p.nc_x, p.nc_y = int(nc), int(ncy or nc)
    p.nf_x, p.nf_y = int(nf), int(nfy or nf)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.feedback = 1 if feedback else 0
    return p, b


class Batch:
    """Many phase-diagram points advanced together on the current CUDA device.

    points: list of dicts with keys t, tp, mu, U, bonds, nc, nf (and
    optionally feedback); all points share one tensor-core precision.  States
    and loops are packed float64 CUDA tensors (1-D); ``view(x, i)`` gives
    point i's [3 or 2][Nl][Nff][Nff] view.
    """

    def __init__(self, points, precision="bf16x3"):
        made = [make_params(q["t"], q["tp"], q["mu"], q["U"], q["bonds"], q["nc"], q["nf"],
                            precision, q.get("feedback", True)) for q in points]
        arr = (_abi.tufrg_params * len(made))(*[m[0] for m in made])
        self._keep = [m[1] for m in made]
        self.n = len(made)
        self.b = _abi.tufrg_batch_setup(arr, _stream())
        self.dims = [_abi.tufrg_batch_dims(self.b, i) for i in range(self.n)]
        _, _, self.state_elems, self.loop_elems = _abi.tufrg_batch_dims(self.b, -1)

    def empty(self, loops=False):
        import torch
        return torch.empty(self.loop_elems if loops else self.state_elems, dtype=torch.float64,
                           device="cuda")

    def zeros(self, loops=False):
        return self.empty(loops).zero_()

    def view(self, x, i, loops=False):
        nl, nff, so, lo = self.dims[i]
        lead = 2 if loops else 3
        off = lo if loops else so
        return x[off:off + lead * nl * nff * nff].view(lead, nl, nff, nff)

    def _vec(self, x, loops=False):
        import torch
        n = self.loop_elems if loops else self.state_elems
        if (not isinstance(x, torch.Tensor) or x.dtype != torch.float64 or not x.is_cuda
                or not x.is_contiguous() or x.numel() != n):
            raise ValueError(f"expected a contiguous float64 CUDA tensor of {n} elements")
        return x.data_ptr()

    def _lams(self, lam):
        lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), (self.n,))
        return np.ascontiguousarray(lam)

    def loops(self, lam, out=None):
        out = self.empty(True) if out is None else out
        _abi.tufrg_batch_loops(self.b, self._lams(lam), self._vec(out, True), _stream())
        return out

    def rhs(self, lam, y, out=None):
        out = self.empty() if out is None else out
        _abi.tufrg_batch_rhs(self.b, self._lams(lam), self._vec(y), self._vec(out), _stream())
        return out

    def flow(self, y=None, lambda0=10.0, lambda_min=1e-3, threshold=50.0, rtol=1e-8,
             atol=1e-10, h0=0.05, max_steps=100000):
        """Flows of every point (DoPri5) in place of y; returns (y, results, statuses)."""
        y = self.zeros() if y is None else y
        o = _abi.tufrg_flow_opts()
        o.lambda0, o.lambda_min, o.threshold = float(lambda0), float(lambda_min), float(threshold)
        o.rtol, o.atol, o.h0 = float(rtol), float(atol), float(h0)
        o.method = TUFRG_DOPRI5
        o.max_steps = int(max_steps)
        o.n_checkpoints = 0
        o.fp64_above = 0.0
        _, res, st = _abi.tufrg_batch_flow(self.b, self.n, o, self._vec(y), _stream())
        return y, [Solver._result(r) for r in res], st

    def attach_surrogate(self, surrogate, judge_every=8, tol=1e-3):
        """Flows use the surrogate's loops while the exact judge accepts them."""
        _abi.tufrg_surrogate_attach(self.ctx, surrogate.s if surrogate else None,
                                    int(judge_every), float(tol))

    def autotune(self, lam=1.0):
        return _abi.tufrg_batch_autotune(self.b, float(lam), _stream()).as_dict()

    def profile_loops(self, lam=0.5, n=3):
        """(contraction kernel ms, loop stage ms) over all points."""
        return _abi.tufrg_batch_profile_loops(self.b, float(lam), int(n), _stream())

    def check(self):
        _abi.tufrg_batch_check(self.b, _stream())

    def close(self):
        if getattr(self, "b", None) is not None:
            _abi.tufrg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """Learned loop surrogate (see include/tufrg.h): an MLP from
    (l_x, l_y, ln Lambda, t', mu) to Lambda (1 + Lambda) chi_dot of the
    parity-allowed pairs of both loops, trained on the GPU."""

    def __init__(self, n_out, width=256, depth=4, seed=1604):
        self.n_out, self.width, self.depth = int(n_out), int(width), int(depth)
        self.s = _abi.tufrg_surrogate_create(self.n_out, self.width, self.depth, int(seed))
        self.n_params = _abi.tufrg_surrogate_n_params(self.s)

    @property
    def sizes(self):
        return [25] + [self.width] * self.depth + [self.n_out]  # after the fixed embedding

    def params(self):
        return _abi.tufrg_surrogate_get_params(self.s, _stream())

    def set_params(self, p):
        _abi.tufrg_surrogate_set_params(self.s, p, _stream())

    def scaling(self):
        """(shift, scale) of the output standardisation."""
        return _abi.tufrg_surrogate_get_scaling(self.s, self.n_out, _stream())

    def set_scaling(self, shift=None, scale=None):
        _abi.tufrg_surrogate_set_scaling(self.s, shift, scale, _stream())

    def samples(self, solver, lam, x=None, t=None):
        """Training rows of one scale from the solver's exact loops:
        (x [Nl][5], t [Nl][n_out]) float32 CUDA tensors (written in place if given)."""
        import torch
        x = torch.empty((solver.nl, 5), dtype=torch.float32, device="cuda") if x is None else x
        t = (torch.empty((solver.nl, self.n_out), dtype=torch.float32, device="cuda")
             if t is None else t)
        _abi.tufrg_surrogate_samples(solver.ctx, self.s, float(lam), x.data_ptr(), t.data_ptr(),
                                     _stream())
        return x, t

    def predict(self, x):
        import torch
        y = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device="cuda")
        _abi.tufrg_surrogate_predict(self.s, x.data_ptr(), int(x.shape[0]), y.data_ptr(),
                                     _stream())
        return y

    def loss_grad(self, x, t):
        return _abi.tufrg_surrogate_loss_grad(self.s, x.data_ptr(), t.data_ptr(),
                                              int(x.shape[0]), _stream())

    def train(self, x, t, epochs=10, batch=4096, lr=1e-3, seed=0):
        return _abi.tufrg_surrogate_train(self.s, x.data_ptr(), t.data_ptr(), int(x.shape[0]),
                                          int(epochs), int(batch), float(lr), int(seed),
                                          _stream())

    def close(self):
        if getattr(self, "s", None) is not None:
            _abi.tufrg_surrogate_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
