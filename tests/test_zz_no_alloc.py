"""The allocation-free loop entry point gives the same loops as the context path.

tufrg_loops_noalloc serves callers that cannot allocate device memory (their
device memory belongs to another allocator, or they hold a fixed budget
reserved at start-up): it works inside one static device array instead of
cudaMalloc'd tables.  Here it is called through the C ABI twice in a row, on
two different problems and scales, and compared with tufrg_loops; a problem
too large for the array must be rejected.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-9


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_noalloc_loops_match_context_loops_on_consecutive_calls():
    import torch
    from paper_1604_06296_gb300 import Solver, TufrgError, _abi, build
    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [  # (shells, nc, nf, t', mu, lambda): two problems, called in a row
        (1, 8, 96, -0.25, -1.0, 0.7),
        (3, 6, 48, -0.35, -1.4, 0.05),
        (1, 8, 96, -0.25, -1.0, 0.05),
    ]
    for shells, nc, nf, tp, mu, lam in cases:
        s = Solver(1.0, tp, mu, 3.0, W.bonds_for_shells(shells), nc, nf)
        ref = s.loops(lam).cpu().numpy()
        out = torch.full((2, s.nl, s.nff, s.nff), float("nan"), dtype=torch.float64,
                         device="cuda")
        _abi.tufrg_loops_noalloc(s.params, lam, out.data_ptr(), stream)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert _rel(got, ref) < RTOL
        s.close()
    # the production fine grid does not fit the static array: rejected, nothing written
    c = W.config("cfg2")
    big = Solver(1.0, -0.25, -1.0, 3.0, W.bonds_for_shells(c["shells"]), c["nc"], c["nf"])
    out = torch.zeros((2, big.nl, big.nff, big.nff), dtype=torch.float64, device="cuda")
    with pytest.raises(TufrgError) as e:
        _abi.tufrg_loops_noalloc(big.params, 0.5, out.data_ptr(), stream)
    assert e.value.status == -1
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0


def test_noalloc_loops_leave_free_device_memory_unchanged():
    """The entry point's defining property: once the library's module is
    loaded (first call), repeated calls change the device's free memory by
    nothing (no cudaMalloc, no allocator of any library)."""
    import torch
    from paper_1604_06296_gb300 import Solver, _abi
    stream = torch.cuda.current_stream().cuda_stream
    s = Solver(1.0, -0.25, -1.0, 3.0, W.bonds_for_shells(1), 8, 96)
    out = torch.empty((2, s.nl, s.nff, s.nff), dtype=torch.float64, device="cuda")
    _abi.tufrg_loops_noalloc(s.params, 0.7, out.data_ptr(), stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for lam in (0.7, 0.05, 2.0):
        _abi.tufrg_loops_noalloc(s.params, lam, out.data_ptr(), stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    s.close()
    assert free1 == free0
