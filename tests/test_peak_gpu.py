"""The measured FP32 peak (fk_peak_fp32) that the bench's roofline fractions divide by:
FFMA chains on every multiprocessor.  It must report the device's multiprocessor count
and a rate that the FP32 lanes can reach: above half, and not above the count of FMA
lanes at the device's highest clock (128 per multiprocessor, 2 flop each)."""
import pytest
import torch

pytestmark = pytest.mark.gpu

fk = pytest.importorskip("paper_2509_02649_b300")


def test_peak_fp32_is_plausible():
    tflops, sms = fk.fk_peak_fp32()
    props = torch.cuda.get_device_properties(0)
    assert sms == props.multi_processor_count
    # highest SM clock: 2032 MHz on B300; allow 2.2 GHz for any part of this family
    ceiling = sms * 128 * 2 * 2.2e9 / 1e12
    assert 0.5 * sms * 128 * 2 * 1.5e9 / 1e12 < tflops <= ceiling


def test_shared_atomic_peak_is_plausible():
    # a warp instruction is at least one shared-memory wavefront, so an SM completes at
    # most 32 lane operations per clock; random windows conflict on banks, so they run
    # slower than windows whose lanes all sit on different banks
    distinct, random = fk.fk_peak_smem_atomics()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 32 * 2.2e9 / 1e9
    assert 0 < random < distinct <= ceiling
