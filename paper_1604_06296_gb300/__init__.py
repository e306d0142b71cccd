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
                 ncy=None, nfy=None):
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
        self.ctx = tufrg_setup(p, _stream())
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

    def close(self):
        if getattr(self, "ctx", None) is not None:
            tufrg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
