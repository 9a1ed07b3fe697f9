"""fgt1d_measure_peaks, the roofline denominators of the FP64 sweeps and the SFU rows:
the rates it measures on the GPU in use must be those of a full device running the
chains (the SM count, an SM clock in range, each pipe's per-clock rate at or below its
nominal issue width and not far under it)."""
import ctypes

import pytest
import torch

from paper_1909_09825_gb300 import _lib

pytestmark = pytest.mark.gpu


def test_measured_pipe_rates(cuda):
    torch.zeros(1, device=cuda)
    o = (ctypes.c_double * 10)()
    assert _lib.lib().fgt1d_measure_peaks(o, None) == _lib.FGT1D_OK
    v = list(o)
    sms, mhz = v[8], v[9]
    assert sms == torch.cuda.get_device_properties(cuda).multi_processor_count
    assert 500 <= mhz <= 2500
    dfma, ffma, ex2, sin = v[1], v[3], v[5], v[7]  # per SM per clock
    assert 0.5 <= dfma <= 2.1        # nominal 2 DFMA per SM per clock
    assert 64 <= ffma <= 128.5       # nominal 128 FFMA per SM per clock
    assert 4 <= ex2 <= 64 and 2 <= sin <= 64
    # operations per second = per-clock rate x SMs x clock
    assert abs(v[0] / (dfma * sms * mhz * 1e6) - 1) < 1e-6
    assert _lib.lib().fgt1d_measure_peaks(None, None) == _lib.FGT1D_EINVAL
