"""Device-side failure detection without a GPU fault: a kernel whose bounded
mbarrier wait can never complete gives up after its poll limit, records a
timeout in the device error word, and returns; hp_stream_status reports
HP_ERR_TIMEOUT, clears the word, and the context keeps working."""
import time

import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_filter_close, rand_volume, to_dev, to_np

pytestmark = pytest.mark.gpu

hp = pytest.importorskip("paper_2511_11890_b300")
from paper_2511_11890_b300 import _lib  # noqa: E402


def test_bounded_wait_reports_timeout_and_context_survives():
    torch.cuda.synchronize()
    hp.stream_status()                       # nothing pending
    t0 = time.perf_counter()
    hp.selftest_wait_timeout()
    with pytest.raises(hp.HPError) as ei:
        hp.stream_status()
    waited = time.perf_counter() - t0
    assert ei.value.status == _lib.HP_ERR_TIMEOUT
    print(f"bounded wait gave up after {waited:.3f} s")
    assert waited < 5.0, "the wait limit should end a stuck wait in about a second"
    hp.stream_status()                       # the word was cleared
    f = rand_volume(np.uint16, (16, 24, 32), 3)
    got = to_np(hp.gaussian3d(to_dev(f), 1.0))
    assert_filter_close(got, oracle.gaussian3d(f, 1.0), "after timeout")
    hp.stream_status()


def test_fp32_fma_probe_is_plausible():
    """The measured FP32 FMA rate lies between a quarter of and just above
    the derived peak (SMs x 128 lanes x 2 flop x max clock)."""
    import torch
    props = torch.cuda.get_device_properties(0)
    rate = hp.probe_fp32_fma(3)
    derived = props.multi_processor_count * 128 * 2 * 2.2e9   # a clock above every B300 boost
    assert 0.25 * derived * (1.9 / 2.2) < rate < 1.05 * derived, rate
    with pytest.raises(hp.HPError):
        hp.probe_fp32_fma(0)
