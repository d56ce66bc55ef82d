"""Failure detection on the GPU without a fault: a bounded wait that nothing
completes runs out of its clock budget, the kernel records it in the handle's
device error word and returns, rtt_device_status reports RTT_ERR_TIMEOUT, and
the same handle then computes correct results."""
import time

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2604_22718_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2604_22718_gb300 import build
    build.build()


def test_bounded_wait_runs_out_and_the_handle_stays_usable():
    from paper_2604_22718_gb300 import rtt
    inst = inputs.make_instance(3, 3, 2, 64, 3.0, seed=8)
    o = orc.Oracle(inst)
    spins = inputs.initial_spins(9, 64, 9)
    with rtt.RTT(inst, "fp16x3", seed=4) as m:
        sg = torch.from_numpy(spins).cuda()
        la0 = m.log_amplitudes(sg)[0]
        assert m.device_status() == (0, 0)
        t0 = time.perf_counter()
        m.wait_selftest(2_000_000)                     # about 1 ms at 2 GHz
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        status, flags = m.device_status()
        assert status == 5 and flags & 1               # RTT_ERR_TIMEOUT, bit 0
        assert m.device_status() == (0, 0)             # cleared by the read
        la1 = m.log_amplitudes(sg)[0]
        e1 = m.local_energy(sg)
        torch.cuda.synchronize()
        assert m.device_status() == (0, 0)
        with pytest.raises(rtt.RTTError, match="INVALID_ARG"):
            m.wait_selftest(10)
    assert dt < 5.0
    assert torch.equal(la0, la1)
    la_o = o.log_amplitudes(spins)[0]
    K = o.amplitude_cond(spins)
    eps = 3 * 2.0 ** -22 + 64 * 2.0 ** -24
    assert np.all(np.abs(la1.cpu().numpy() - la_o) <= eps * (K[:, 0] + K[:, 2]))
    assert np.all(np.isfinite(e1.cpu().numpy()))


def test_wait_selftest_needs_a_tensor_core_handle():
    from paper_2604_22718_gb300 import rtt
    with rtt.RTT(inputs.workload("tiny_fp64"), "fp64") as m:
        with pytest.raises(rtt.RTTError, match="UNSUPPORTED"):
            m.wait_selftest(2_000_000)
