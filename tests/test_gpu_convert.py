"""The library's FP64 <-> FP32 conversions (integer-pipe bit manipulation used
by the FP32 projections and products) equal the GPU's conversion instructions
bit for bit: round to nearest even for FP64 -> FP32 (ties, near ties, the
normal/subnormal boundary, overflow to infinity, zeros of both signs,
infinities, NaN), exact FP32 -> FP64."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs():
    rng = np.random.default_rng(7)
    n = 1 << 20
    x = rng.standard_normal(n) * 10.0 ** rng.integers(-46, 40, n)
    f = (rng.standard_normal(8192) * 10.0 ** rng.integers(-37, 38, 8192)).astype(np.float32)
    lo = f.astype(np.float64)
    hi = np.nextafter(f, np.float32(np.inf)).astype(np.float64)
    mid = (lo + hi) / 2  # exact ties of FP32 rounding
    special = [0.0, -0.0, 3.4028234663852886e38, 3.4028235677973366e38, 3.402823567797337e38,
               1e39, -1e39, 1.1754943508222875e-38, 1.1754942106924411e-38, 1e-40, 5e-324,
               np.inf, -np.inf, np.nan, 1.0, -1.0, 0.5 * (1 + 2.0 ** -24), 1 + 2.0 ** -23]
    return np.concatenate([x, mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf),
                           np.array(special)])


def test_conversions_equal_the_hardware_bit_for_bit():
    import torch
    from paper_1604_06296_gb300 import _abi, build
    build.build()
    x = torch.from_numpy(_inputs()).cuda()
    y32 = torch.empty(x.numel(), dtype=torch.float32, device="cuda")
    back = torch.empty_like(x)
    _abi.tufrg_selftest_convert(x.data_ptr(), y32.data_ptr(), back.data_ptr(), x.numel(),
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ref32 = x.to(torch.float32)
    nan = torch.isnan(x)
    assert torch.equal(torch.isnan(y32), nan)
    assert torch.equal(y32[~nan].view(torch.int32), ref32[~nan].view(torch.int32))
    ref64 = y32.to(torch.float64)
    assert torch.equal(torch.isnan(back), nan)
    assert torch.equal(back[~nan].view(torch.int64), ref64[~nan].view(torch.int64))


def test_conversion_rejects_bad_arguments():
    import torch
    from paper_1604_06296_gb300 import TufrgError, _abi
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    y = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(TufrgError):
        _abi.tufrg_selftest_convert(x.data_ptr(), y.data_ptr(), x.data_ptr(), -1)
    with pytest.raises(TufrgError):
        _abi.tufrg_selftest_convert(0, y.data_ptr(), x.data_ptr(), 4)
