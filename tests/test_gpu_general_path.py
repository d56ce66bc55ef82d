"""General paths (orderings sigma^V, sigma^H, sigma^D, sigma^D' one after the
other, Sec. 2.2.1 and Sec. 4) on the SIMT sampler: FP64 bit-exact against the
oracle, FP32 within its tolerance at the full vhdd_6x6 size."""
import math

import numpy as np
import pytest
import torch

from paper_2604_22718_gb300 import inputs
from parity_util import check_sweep_divergences, eps_site
from oracle import oracle as orc
from oracle import dual

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _rtt():
    from paper_2604_22718_gb300 import rtt
    return rtt


CASES = [(3, 3, ("V", "H", "D", "Dp"), 8), (4, 4, ("H", "V"), 16), (3, 4, ("D", "Dp", "V"), 5)]


@pytest.mark.parametrize("lx,ly,names,chi", CASES)
def test_fp64_amplitudes_energies_ratios_bit_exact(lx, ly, names, chi):
    rtt = _rtt()
    inst = inputs.make_path_instance(lx, ly, names, chi, 3.0, seed=31)
    o = orc.Oracle(inst)
    B = 211
    spins = inputs.initial_spins(32, B, lx * ly)
    la_o, sg_o, _, _ = o.log_amplitudes(spins)
    e_o, r_o = o.local_energies(spins, with_ratios=True, threads=8)
    with rtt.RTT(inst, "fp64") as m:
        sp = torch.from_numpy(spins).cuda()
        la, sg, _ = m.log_amplitudes(sp)
        e, r = m.local_energy(sp, with_ratios=True)
        torch.cuda.synchronize()
    assert np.array_equal(la.cpu().numpy(), la_o) and np.array_equal(sg.cpu().numpy(), sg_o)
    assert np.array_equal(e.cpu().numpy(), e_o)
    assert np.array_equal(r.cpu().numpy(), r_o)


@pytest.mark.parametrize("lx,ly,names,chi", CASES[:2])
def test_fp64_chains_bit_exact(lx, ly, names, chi):
    rtt = _rtt()
    inst = inputs.make_path_instance(lx, ly, names, chi, 3.0, seed=33)
    o = orc.Oracle(inst)
    B, n_sw = 64, 4
    s0 = inputs.initial_spins(34, B, lx * ly)
    so = s0.copy()
    mo, eo = o.init_chains(so)
    tr_o, acc_o = o.mcmc(77, so, mo, eo, 3, n_sw, measure_every=2, threads=8)
    with rtt.RTT(inst, "fp64", seed=77) as m:
        sg = torch.from_numpy(s0.copy()).cuda()
        _, _, st = m.log_amplitudes(sg)
        tr = torch.empty((2, B), dtype=torch.float64, device="cuda")
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        m.mcmc_sweep(sg, st, 3, n_sw, 2, tr, acc)
        torch.cuda.synchronize()
    assert np.array_equal(sg.cpu().numpy(), so)
    assert np.array_equal(acc.cpu().numpy(), acc_o)
    assert np.array_equal(tr.cpu().numpy(), tr_o)
    st = st.cpu().numpy()
    assert np.array_equal(st[:, 0].view(np.float64), mo) and np.array_equal(st[:, 1], eo)


def test_fp32_vhdd_6x6_full_batch_sampled():
    rtt = _rtt()
    w = inputs.WORKLOADS["vhdd_6x6"]
    inst = inputs.workload("vhdd_6x6")
    o = orc.Oracle(inst)
    B = w["chains"]
    s0 = inputs.initial_spins(w["seed"], B, 36)
    pick = np.array([0, 7, 2048, B - 1])
    with rtt.RTT(inst, "fp32", seed=w["seed"]) as m:
        sg = torch.from_numpy(s0.copy()).cuda()
        la, _, st = m.log_amplitudes(sg)
        e = m.local_energy(sg)
        tr = torch.empty((2, B), dtype=torch.float64, device="cuda")
        m.mcmc_sweep(sg, st, 0, 2, 1, tr)
        torch.cuda.synchronize()
        s_now = sg.cpu().numpy()
    la, e, tr = la.cpu().numpy(), e.cpu().numpy(), tr.cpu().numpy()
    la_o = o.log_amplitudes(s0[pick])[0]
    kfin = o.amplitude_cond(s0[pick])[:, 2]
    tol = 1e-5 * np.maximum(1.0, np.abs(la_o)) + 2 * U32 * math.sqrt(o.L) * kfin
    assert np.all(np.abs(la[pick] - la_o) <= tol)
    e_o = o.local_energies(s0[pick], threads=4)
    np.testing.assert_allclose(e[pick], e_o, rtol=2e-5, atol=2e-5 * (inst.bonds.shape[0] + 3.0 * 36))
    np.testing.assert_allclose(tr[0][pick], e[pick], rtol=0, atol=0)   # entering configuration
    assert np.all(np.isfinite(tr)) and s_now.shape == s0.shape


def test_mixed_energy_between_periodic_and_general_paths_bit_exact():
    rtt = _rtt()
    a = inputs.make_instance(3, 3, 2, 6, 3.0, seed=35)
    b = inputs.make_path_instance(3, 3, ("V", "H"), 6, 3.0, seed=36)
    spins = inputs.initial_spins(37, 150, 9)
    e_o, r_o = dual.mixed_local_energies(orc.Oracle(a), orc.Oracle(b), spins)
    with rtt.RTT(a, "fp64") as ma, rtt.RTT(b, "fp64") as mb:
        e, r = ma.mixed_local_energy(mb, torch.from_numpy(spins).cuda())
        torch.cuda.synchronize()
    assert np.array_equal(e.cpu().numpy(), e_o) and np.array_equal(r.cpu().numpy(), r_o)


def test_general_path_rejected_where_unsupported():
    rtt = _rtt()
    with pytest.raises(rtt.RTTError):
        rtt.RTTBatch([inputs.make_path_instance(6, 6, ("V", "H"), 32, 3.0, seed=39)], [8])


# ---------------------------------------------------------------- tensor cores

UB16 = 2.0 ** -11


def _eps_site(chi):
    return 3 * UB16 ** 2 + chi * U32


@pytest.mark.parametrize("lx,ly,names,chi,B", [(6, 6, ("V", "H", "D", "Dp"), 64, 300),
                                               (4, 4, ("H", "D", "V"), 128, 140)])
def test_fp16x3_general_path_amplitudes_and_energies(lx, ly, names, chi, B):
    """Split-precision amplitudes within eps_site (sum kappa_k + kappa_fin) of
    the oracle; every flip ratio within |r| eps_site (K(s) + K(s^(i))); the mean
    local energy within 1e-4 relative (the metric's gate)."""
    rtt = _rtt()
    inst = inputs.make_path_instance(lx, ly, names, chi, 3.0, seed=61)
    o = orc.Oracle(inst)
    n = lx * ly
    spins = inputs.initial_spins(62, B, n)
    la_o = o.log_amplitudes(spins)[0]
    nc = 24
    e_o, r_o = o.local_energies(spins[:nc], with_ratios=True, threads=16)
    with rtt.RTT(inst, "fp16x3") as m:
        sp = torch.from_numpy(spins).cuda()
        la = m.log_amplitudes(sp)[0].cpu().numpy()
        e, r = m.local_energy(sp[:nc].contiguous(), with_ratios=True)
        torch.cuda.synchronize()
    e, r = e.cpu().numpy(), r.cpu().numpy()
    eps = _eps_site(chi)
    K = o.amplitude_cond(spins)
    assert np.all(np.abs(la - la_o) <= eps * (K[:, 0] + K[:, 2]))
    flipped = np.repeat(spins[:nc], n, axis=0)
    flipped[np.arange(nc * n), np.tile(np.arange(n), nc)] ^= 1
    Kf = o.amplitude_cond(flipped)
    Kf = (Kf[:, 0] + Kf[:, 2]).reshape(nc, n)
    bound = np.abs(r_o) * eps * ((K[:nc, 0] + K[:nc, 2])[:, None] + Kf)
    assert np.all(np.abs(r - r_o) <= bound)
    rel_mean = abs(e.mean() - e_o.mean()) / max(abs(e_o.mean()), np.mean(np.abs(e_o)))
    assert rel_mean <= 1e-4, rel_mean


@pytest.mark.parametrize("case", ["vhdd_6x6_chi64", "vh_4x4_chi128"])
def test_fp16x3_general_path_sweep_follows_oracle(case):
    """The general split-row sweeps on CTA pairs (chi = 64 dense, sigma^V +
    sigma^H + sigma^D + sigma^D', three row tiles; chi = 128 sparse, sigma^V +
    sigma^H, two row tiles): every decision of one sweep is the FP64 rule's at
    the same state except at explained near ties; tracked amplitudes stay those
    of the spins; the measured trace is the standalone energy of the entering
    configurations."""
    rtt = _rtt()
    if case == "vhdd_6x6_chi64":
        inst, B = inputs.workload("vhdd_6x6"), 300
    else:
        inst, B = inputs.make_path_instance(4, 4, ("V", "H"), 128, 3.0, seed=38), 200
    o = orc.Oracle(inst)
    s0 = inputs.initial_spins(63, B, inst.n_spins)
    with rtt.RTT(inst, "fp16x3", seed=17) as m:
        sg = torch.from_numpy(s0.copy()).cuda()
        _, _, st = m.log_amplitudes(sg)
        e0 = m.local_energy(sg)
        tr = torch.empty((1, B), dtype=torch.float64, device="cuda")
        m.mcmc_sweep(sg, st, 0, 1, 1, tr)
        la_track = (rtt.state_exp(st).double() * math.log(2) +
                    torch.log(rtt.state_mant(st).abs())).cpu().numpy()
        la_now = m.log_amplitudes(sg)[0].cpu().numpy()
        torch.cuda.synchronize()
    s1 = sg.cpu().numpy()
    eps = eps_site(inst.chi, "fp16x3")
    n, nd, worst = check_sweep_divergences(o, 17, s0, s1, 0, eps, slack=2.0 ** -23)
    print(f"general path sweep: {nd} of {n} decisions differ, worst gap/tolerance {worst:.3f}")
    d = np.abs(la_track - la_now)
    K = o.amplitude_cond(s1)
    assert np.all(d <= 2 * eps * (K[:, 0] + K[:, 2]))
    assert torch.equal(tr[0], e0)
