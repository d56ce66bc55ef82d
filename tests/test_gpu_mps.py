"""R = 1: the RTT is a matrix product state (Sec. 2.1), whose energy the
oracle computes exactly in polynomial time by transfer matrices.  The GPU
samplers' Monte Carlo mean of the local energy on the 6x6 lattice (N = 36)
at chi = 64 must agree with it within 3 standard errors: FP64 and FP32 on
the CUDA cores and FP16X3 on the tensor cores (the tile kernel's sweep, which
R = 1 paths take)."""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16x3"])
def test_r1_sampler_mean_matches_transfer_matrix_energy(prec):
    from paper_2604_22718_gb300 import rtt
    inst = inputs.make_instance(6, 6, 1, 64, 3.0, seed=77, mixing=True)
    e_exact = orc.mps_energy(inst)
    B, burn, T = 4096, 40, 200
    with rtt.RTT(inst, prec, seed=78) as m:
        sg = torch.from_numpy(inputs.initial_spins(79, B, 36)).cuda()
        _, _, st = m.log_amplitudes(sg)
        m.mcmc_sweep(sg, st, 0, burn)
        tr = torch.empty((T, B), dtype=torch.float64, device="cuda")
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        m.mcmc_sweep(sg, st, burn, T, 1, tr, acc)
        obs = m.observables(tr, acc, T * 36)
        if prec == "fp16x3":
            flags = rtt.ctypes.c_int32()
            assert rtt.lib().rtt_device_status(m.handle, rtt.ctypes.byref(flags)) == 0
    print(prec, "MC", obs["mean"], "+-", obs["se"], "(tau", obs["tau_int"], ") transfer matrix", e_exact)
    assert np.isfinite(obs["mean"]) and obs["se"] > 0
    assert abs(obs["mean"] - e_exact) < 3.0 * obs["se"], (obs, e_exact)
    assert 0.0 < obs["accept_rate"] < 1.0
