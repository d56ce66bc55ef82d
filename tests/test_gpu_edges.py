"""Edge cases and full sizes not covered elsewhere: the largest bond dimension
(and a padded one) on the SIMT path, tensor-core sweeps over several row tiles
with a ragged last tile, and the headline FP16X3 configuration at its full 4096
chains sampled against the oracle."""
import math

import numpy as np
import pytest
import torch

from paper_2604_22718_gb300 import inputs
from oracle import oracle as orc
from parity_util import check_sweep_divergences, eps_site, local_energy_bound

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _rtt():
    from paper_2604_22718_gb300 import rtt
    return rtt


def _status_ok(rtt, m):
    flags = rtt.ctypes.c_int32()
    return rtt.lib().rtt_device_status(m.handle, rtt.ctypes.byref(flags)) == 0 and flags.value == 0


@pytest.mark.parametrize("chi", [256, 200])
def test_simt_largest_bond_dimension(chi):
    rtt = _rtt()
    inst = inputs.make_instance(2, 3, 2, chi, 3.0, seed=40 + chi)
    o = orc.Oracle(inst)
    B = 37
    spins = inputs.initial_spins(41, B, 6)
    la_o, sg_o, _, _ = o.log_amplitudes(spins)
    e_o, r_o = o.local_energies(spins, with_ratios=True)
    with rtt.RTT(inst, "fp64") as m:
        sp = torch.from_numpy(spins).cuda()
        la, sg, _ = m.log_amplitudes(sp)
        e, r = m.local_energy(sp, with_ratios=True)
        torch.cuda.synchronize()
    assert np.array_equal(la.cpu().numpy(), la_o) and np.array_equal(sg.cpu().numpy(), sg_o)
    assert np.array_equal(e.cpu().numpy(), e_o) and np.array_equal(r.cpu().numpy(), r_o)
    with rtt.RTT(inst, "fp32") as m:
        la32 = m.log_amplitudes(torch.from_numpy(spins).cuda())[0].cpu().numpy()
    kfin = o.amplitude_cond(spins)[:, 2]
    tol = 1e-5 * np.maximum(1.0, np.abs(la_o)) + 2 * U32 * math.sqrt(o.L) * kfin
    assert np.all(np.abs(la32 - la_o) <= tol)


@pytest.mark.parametrize("chi,B", [(64, 300), (128, 200)])
def test_tc_sweep_ragged_tiles_follow_oracle(chi, B):
    """Several 128-row tiles and a ragged last one: every decision of one
    FP16X3 sweep is the FP64 rule's at the same state except at explained near
    ties; every chain's amplitude stays consistent with its spins."""
    rtt = _rtt()
    inst = inputs.make_instance(4, 4, 2, chi, 3.0, seed=50 + chi)
    o = orc.Oracle(inst)
    s0 = inputs.initial_spins(51, B, 16)
    with rtt.RTT(inst, "fp16x3", seed=13) as m:
        sg = torch.from_numpy(s0.copy()).cuda()
        _, _, st = m.log_amplitudes(sg)
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        m.mcmc_sweep(sg, st, 0, 1, 1, None, acc)
        la_track = (rtt.state_exp(st).double() * math.log(2) +
                    torch.log(rtt.state_mant(st).abs())).cpu().numpy()
        la_now = m.log_amplitudes(sg)[0].cpu().numpy()
        torch.cuda.synchronize()
        assert _status_ok(rtt, m)
    s1 = sg.cpu().numpy()
    n, nd, worst = check_sweep_divergences(o, 13, s0, s1, 0, eps_site(chi, "fp16x3"),
                                           slack=2.0 ** -23)
    print(f"chi {chi}: {nd} of {n} decisions differ, worst gap/tolerance {worst:.3f}")
    # the tracked amplitude of every chain (last tile included) is its spins' amplitude
    d = np.abs(la_track - la_now)
    K = o.amplitude_cond(s1)
    assert np.all(d <= 2 * eps_site(chi, "fp16x3") * (K[:, 0] + K[:, 2])), np.sort(d)[-5:]
    assert np.all(acc.cpu().numpy() == np.sum(s1 != s0, axis=1))


def test_plain_6x6_fp16x3_full_batch_sampled():
    """The 6x6 configuration: 4096 chains, FP16X3, two measured sweeps (two
    calls); for picked chains the measured energies of the entering
    configurations and the final local energies against the oracle on the
    same configurations, each within its own split bound, and both sweeps'
    decisions replayed by the oracle, every divergence an explained near tie."""
    rtt = _rtt()
    w = inputs.WORKLOADS["plain_6x6"]
    inst = inputs.workload("plain_6x6")
    o = orc.Oracle(inst)
    B = w["chains"]
    s0 = inputs.initial_spins(w["seed"], B, 36)
    pick = np.array([0, 1, 127, 128, 2047, 4000, B - 1])
    with rtt.RTT(inst, "fp16x3", seed=w["seed"]) as m:
        sg = torch.from_numpy(s0.copy()).cuda()
        _, _, st = m.log_amplitudes(sg)
        tr = torch.empty((2, B), dtype=torch.float64, device="cuda")
        m.mcmc_sweep(sg, st, 0, 1, 1, tr[0:1])
        s1 = sg.cpu().numpy()
        m.mcmc_sweep(sg, st, 1, 1, 1, tr[1:2])
        e_end, r_end = m.local_energy(sg, with_ratios=True)
        torch.cuda.synchronize()
        assert _status_ok(rtt, m)
        s2 = sg.cpu().numpy()
    tr, e_end = tr.cpu().numpy(), e_end.cpu().numpy()
    eps = eps_site(64, "fp16x3")
    for a, b, sweep in ((s0, s1, 0), (s1, s2, 1)):
        for c in pick:
            check_sweep_divergences(o, w["seed"], a[c:c + 1], b[c:c + 1], sweep, eps,
                                    chain0=int(c), slack=2.0 ** -23)
    for conf, e_gpu in ((s0, tr[0]), (s1, tr[1]), (s2, e_end)):
        e_o, r_o = o.local_energies(conf[pick], with_ratios=True, threads=7)
        bound = local_energy_bound(o, conf[pick], r_o, eps, inst.J, inst.h, inst.bonds.shape[0])
        assert np.all(np.abs(e_gpu[pick] - e_o) <= bound), (e_gpu[pick], e_o, bound)
