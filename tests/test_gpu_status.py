"""The bounded device-side waits: a wait that runs out is reported through the
device status word, and the CUDA context stays usable afterwards.

The self-test kernel waits on an mbarrier that nothing completes, so its wait
must give up after the requested time; no memory is touched and nothing hangs.
"""
import numpy as np
import pytest
import torch

import paper_1710_08332_gb300 as dpia
from paper_1710_08332_gb300 import _native as N
from oracle import loopnest
from synth import workloads as W
from tests.helpers import assert_bits_equal, host, oracle_strategy

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(cuda_device):
    assert dpia.dpia_poll_device_status() == 0
    dpia.dpia_selftest_bounded_wait(2000)  # 2 ms
    torch.cuda.synchronize()
    assert dpia.dpia_poll_device_status() == N.ERR_TIMEOUT
    assert dpia.dpia_poll_device_status() == 0  # the poll cleared the flag
    # the context still runs the staged reduction (whose waits complete)
    x, y = W.dot_f32("cuda", n=(1 << 18) + 5, seed=9)
    st = dpia.ReduceStrategy(split=8192, threads=256, vec=4, pad=True, stage="local")
    got = dpia.dot(x, y, st)
    torch.cuda.synchronize()
    assert_bits_equal(np.float32(host(got)), loopnest.dot_f32(host(x), host(y), oracle_strategy(st)), "after")
    assert dpia.dpia_poll_device_status() == 0
