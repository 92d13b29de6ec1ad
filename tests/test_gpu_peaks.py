"""The peak microbenchmarks (roofline denominators) through the C ABI: each rate is positive and
bounded by what the device's units and the clock the run reports allow."""
import pytest
import torch

from paper_1306_2258_gb300 import _lib

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_physical():
    assert torch.cuda.is_available()
    m = _lib.sas_measure_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = m["sm_mhz"]
    assert 500.0 < mhz < 2500.0
    lanes = sms * 128 * mhz * 1e6                    # FP32 lanes x clock
    for k in ("ffma", "ffma2"):
        assert 0.5 * lanes < m[k] <= 1.05 * lanes, (k, m[k], lanes)
    # three distinct source operands per packed FMA: no faster than the packed rate with shared ones
    assert 0.25 * lanes < m["ffma2_3op"] <= 1.05 * m["ffma2"], (m["ffma2_3op"], m["ffma2"])
    assert 0.0 < m["mufu_sin"] <= 0.3 * lanes        # MUFU: a fraction of the FP32 rate
    assert 0.0 < m["dfma"] <= 0.1 * lanes            # FP64 is a small fraction on this part
    assert 0.0 < m["atoms_shared"] <= 0.25 * lanes   # at most one 32-lane atomic per SM clock
