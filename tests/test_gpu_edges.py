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
    """Several 128-row tiles and a ragged last one: one FP16X3 sweep takes the
    oracle's decisions on at least 90 % of the chains (the rest are near ties),
    every chain's amplitude stays consistent with its spins."""
    rtt = _rtt()
    inst = inputs.make_instance(4, 4, 2, chi, 3.0, seed=50 + chi)
    o = orc.Oracle(inst)
    s0 = inputs.initial_spins(51, B, 16)
    so = s0.copy()
    mo, eo = o.init_chains(so)
    o.mcmc(13, so, mo, eo, 0, 1, record=False, threads=16)
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
    same = np.all(sg.cpu().numpy() == so, axis=1)
    assert same.mean() >= 0.9, same.mean()
    # the tracked amplitude of every chain (last tile included) is its spins' amplitude
    d = np.abs(la_track - la_now)
    assert np.median(d) < 1e-5 and np.mean(d <= 1e-3) >= 0.99, np.sort(d)[-5:]
    assert np.all(acc.cpu().numpy() <= 16)


def test_plain_6x6_fp16x3_full_batch_sampled():
    """The bench configuration: 4096 chains, FP16X3, two measured sweeps; sampled
    chains' measured energies (entering configurations) against the oracle on
    the seeded start, and the final local energies against the oracle's own
    chains where the two took the same steps."""
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
        m.mcmc_sweep(sg, st, 0, 2, 1, tr)
        e_end = m.local_energy(sg)
        torch.cuda.synchronize()
        assert _status_ok(rtt, m)
        s_end = sg.cpu().numpy()
    tr, e_end = tr.cpu().numpy(), e_end.cpu().numpy()
    scale = inst.bonds.shape[0] + inst.h * 36
    e0_o = o.local_energies(s0[pick], threads=7)
    assert np.all(np.abs(tr[0][pick] - e0_o) <= 1e-3 * scale), (tr[0][pick], e0_o)
    # the final energies on the oracle's own chains (each picked chain run alone
    # under its own chain index), where the FP16X3 chains took the same steps
    so = s0[pick].copy()
    for k, c in enumerate(pick):
        sc = s0[c:c + 1].copy()
        mc, ec = o.init_chains(sc)
        o.mcmc(w["seed"], sc, mc, ec, 0, 2, chain0=int(c), record=False)
        so[k] = sc[0]
    same = np.all(s_end[pick] == so, axis=1)
    e_o = o.local_energies(so, threads=7)
    assert np.all((np.abs(e_end[pick] - e_o) <= 1e-3 * scale)[same]), (e_end[pick], e_o, same)
