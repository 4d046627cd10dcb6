"""The float64 FMA-rate probe (mg_fp64_fma_peak), through the C ABI.

The outer Krylov operator is bound by the float64 FMA rate; bench.py reports
this probe's rate (a lower bound on the float64 pipe's) beside the peak
derived from unit counts and the SM clock.  The check here is that the probe
runs and returns a rate between a tenth of a TFLOP/s and what the widest
float64 pipe (64 FMAs per clock per SM) could reach at 3 GHz.
"""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fp64_fma_peak_is_plausible(gpu_lib):
    from paper_1604_07163_gb300 import _lib
    lib = _lib.load()
    r = ctypes.c_double()
    assert lib.mg_fp64_fma_peak(3, ctypes.byref(r)) == 0
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert 0.1 < r.value < nsm * 128 * 3.0e9 / 1e12, r.value
