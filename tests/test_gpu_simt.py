"""GPU parity of the SIMT paths (FP64, FP32) against the FP64 oracle, through
the C ABI.  FP64 must reproduce the oracle bit for bit (same canonical fma
order, same exact power-of-two rescaling, same Philox stream); FP32 must stay
within the tolerances stated per test."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2604_22718_gb300 import inputs
from parity_util import check_sweep_divergences, eps_site

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24   # FP32 unit roundoff


def fp32_logpsi_tol(o, spins, la_o):
    """Tolerance of an FP32 log|psi|: 1e-5 relative (floor 1), plus the
    componentwise rounding of the row after L sites (a random walk of about
    u32 per site, sqrt(L) u32) amplified by the closing contraction's
    condition number kappa_fin = sum|v_b b_R,b| / |v . b_R| (oracle, FP64)."""
    kfin = o.amplitude_cond(spins)[:, 2]
    return 1e-5 * np.maximum(1.0, np.abs(la_o)) + 2 * U32 * math.sqrt(o.L) * kfin


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2604_22718_gb300 import build
    build.build()


def _rtt():
    from paper_2604_22718_gb300 import rtt
    return rtt


def _inst(lx, ly, R, chi, seed, h=3.0, mixing=True):
    return inputs.make_instance(lx, ly, R, chi, h, seed=seed, mixing=mixing)


CASES = [
    ("tiny_fp64", lambda: inputs.workload("tiny_fp64"), 100),
    ("6x6_R2_chi64", lambda: _inst(6, 6, 2, 64, 5), 37),
    ("2x3_R3_chi3_padded", lambda: _inst(2, 3, 3, 3, 6), 70),
    ("4x4_R1_chi16_mps", lambda: _inst(4, 4, 1, 16, 7), 33),
    ("3x3_R2_chi1", lambda: _inst(3, 3, 2, 1, 8, mixing=False), 65),
    ("3x4_R4_chi24_padded", lambda: _inst(3, 4, 4, 24, 9), 41),
]


def _state_np(rtt, st):
    return rtt.state_mant(st).cpu().numpy(), rtt.state_exp(st).cpu().numpy()


# ---------------------------------------------------------------- RNG

def test_device_uniforms_match_numpy_philox():
    rtt = _rtt()
    rng = np.random.default_rng(0)
    ctr = np.stack([rng.integers(1, 2**40, 300), rng.integers(0, 2**20, 300),
                    rng.integers(0, 600, 300)], axis=1).astype(np.int64)
    got = rtt.mcmc_uniforms(22720, torch.from_numpy(ctr).cuda()).cpu().numpy()
    for k in range(ctr.shape[0]):
        c = [int(ctr[k, 0]) - 1, int(ctr[k, 1]), int(ctr[k, 2]), 0]
        bg = np.random.Philox(counter=np.array(c, np.uint64), key=np.array([22720, 0x4D434D43], np.uint64))
        x0 = int(bg.random_raw(1)[0])
        assert got[k] == float(x0 >> 11) * 2.0 ** -53


# ---------------------------------------------------------------- amplitudes

@pytest.mark.parametrize("name,make,B", CASES, ids=[c[0] for c in CASES])
def test_fp64_log_amplitudes_bit_exact(name, make, B):
    rtt = _rtt()
    inst = make()
    o = orc.Oracle(inst)
    spins = inputs.initial_spins(11, B, inst.n_spins)
    la_o, sg_o, m_o, e_o = o.log_amplitudes(spins)
    with rtt.RTT(inst, "fp64") as m:
        la, sg, st = m.log_amplitudes(torch.from_numpy(spins).cuda())
        mm, ee = _state_np(rtt, st)
    assert np.array_equal(mm, m_o) and np.array_equal(ee, e_o)
    assert np.array_equal(sg.cpu().numpy(), sg_o)
    np.testing.assert_allclose(la.cpu().numpy(), la_o, rtol=1e-14, atol=0)


@pytest.mark.parametrize("name,make,B", CASES, ids=[c[0] for c in CASES])
def test_fp32_log_amplitudes_within_1e5(name, make, B):
    rtt = _rtt()
    inst = make()
    o = orc.Oracle(inst)
    spins = inputs.initial_spins(12, B, inst.n_spins)
    la_o, sg_o, _, _ = o.log_amplitudes(spins)
    with rtt.RTT(inst, "fp32") as m:
        la, sg, _ = m.log_amplitudes(torch.from_numpy(spins).cuda())
    la, sg = la.cpu().numpy(), sg.cpu().numpy()
    err = np.abs(la - la_o)
    plain = 1e-5 * np.maximum(1.0, np.abs(la_o))
    tol = fp32_logpsi_tol(o, spins, la_o)
    print(f"[{name}] fp32 log|psi|: max err {err.max():.2e}, within plain 1e-5: "
          f"{np.mean(err <= plain):.3f}")
    assert np.all(err <= tol), np.max(err / tol)
    assert np.mean(err <= plain) >= 0.9
    assert np.array_equal(sg, sg_o)


# ---------------------------------------------------------------- local energy

@pytest.mark.parametrize("name,make,B", CASES, ids=[c[0] for c in CASES])
def test_fp64_local_energy_and_ratios_bit_exact(name, make, B):
    rtt = _rtt()
    inst = make()
    o = orc.Oracle(inst)
    B = min(B, 20)
    spins = inputs.initial_spins(13, B, inst.n_spins)
    e_o, r_o = o.local_energies(spins, with_ratios=True, threads=8)
    with rtt.RTT(inst, "fp64") as m:
        e, r = m.local_energy(torch.from_numpy(spins).cuda(), with_ratios=True)
    assert np.array_equal(r.cpu().numpy(), r_o)
    assert np.array_equal(e.cpu().numpy(), e_o)


@pytest.mark.parametrize("name,make,B", CASES, ids=[c[0] for c in CASES])
def test_fp32_local_energy(name, make, B):
    """|dE| <= 2e-5 * (|J| n_bonds + |h| sum_i |ratio_i|): per-ratio FP32
    error of a few ulps per site over <= (R-1)N+1 sites of unit-scale rows."""
    rtt = _rtt()
    inst = make()
    o = orc.Oracle(inst)
    B = min(B, 20)
    spins = inputs.initial_spins(14, B, inst.n_spins)
    e_o, r_o = o.local_energies(spins, with_ratios=True, threads=8)
    with rtt.RTT(inst, "fp32") as m:
        e, r = m.local_energy(torch.from_numpy(spins).cuda(), with_ratios=True)
    e, r = e.cpu().numpy(), r.cpu().numpy()
    scale = abs(inst.J) * inst.bonds.shape[0] + abs(inst.h) * np.abs(r_o).sum(axis=1)
    assert np.all(np.abs(e - e_o) <= 2e-5 * scale), np.max(np.abs(e - e_o) / scale)
    # ratios enter E_loc additively: bound |d ratio| on the scale max(1, |ratio|)
    span = (inst.path.shape[0] // inst.n_spins - 1) * inst.n_spins + 1
    assert np.all(np.abs(r - r_o) <= (2e-6 * span + 1e-5) * np.maximum(1.0, np.abs(r_o)))


# ---------------------------------------------------------------- Metropolis

def _run_both(inst, B, seed, chain0, sweep0, n_sw, every, prec="fp64", spins_seed=21):
    rtt = _rtt()
    o = orc.Oracle(inst)
    s0 = inputs.initial_spins(spins_seed, B, inst.n_spins)
    so = s0.copy()
    mo, eo = o.init_chains(so)
    tr_o, acc_o = o.mcmc(seed, so, mo, eo, sweep0, n_sw, measure_every=every, chain0=chain0,
                         threads=8)
    with rtt.RTT(inst, prec, seed=seed) as m:
        sg = torch.from_numpy(s0.copy()).cuda()
        _, _, st = m.log_amplitudes(sg)
        nm = n_sw // every
        tr = torch.empty((nm, B), dtype=torch.float64, device="cuda")
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        m.mcmc_sweep(sg, st, sweep0, n_sw, every, tr, acc, chain0=chain0)
        torch.cuda.synchronize()
        mm, ee = _state_np(rtt, st)
        return (so, mo, eo, tr_o, acc_o), (sg.cpu().numpy(), mm, ee, tr.cpu().numpy(), acc.cpu().numpy())


@pytest.mark.parametrize("inst_fn,B,n_sw,every,chain0,sweep0", [
    (lambda: inputs.workload("tiny_fp64"), 64, 6, 1, 0, 0),
    (lambda: inputs.workload("tiny_fp64"), 45, 5, 2, 1000, 77),
    (lambda: _inst(6, 6, 2, 64, 5), 6, 2, 1, 3, 11),
    (lambda: _inst(2, 3, 3, 3, 6), 70, 4, 1, 0, 0),
    (lambda: _inst(4, 4, 1, 16, 7), 33, 3, 3, 0, 5),
], ids=["tiny", "tiny_offsets_every2", "6x6_chi64", "chi3_padded", "R1"])
def test_fp64_chains_bit_exact(inst_fn, B, n_sw, every, chain0, sweep0):
    inst = inst_fn()
    (so, mo, eo, tr_o, acc_o), (sg, mm, ee, tr, acc) = _run_both(inst, B, 22719, chain0, sweep0,
                                                                 n_sw, every)
    assert np.array_equal(sg, so)
    assert np.array_equal(acc, acc_o)
    assert np.array_equal(mm, mo) and np.array_equal(ee, eo)
    assert np.array_equal(tr, tr_o)


def test_fp64_split_calls_reproduce_one_call():
    rtt = _rtt()
    inst = inputs.workload("tiny_fp64")
    s0 = inputs.initial_spins(3, 50, 9)
    outs = []
    with rtt.RTT(inst, "fp64", seed=5) as m:
        for split in (False, True):
            sg = torch.from_numpy(s0.copy()).cuda()
            _, _, st = m.log_amplitudes(sg)
            tr = torch.empty((6, 50), dtype=torch.float64, device="cuda")
            if split:
                m.mcmc_sweep(sg, st, 0, 2, 1, tr[:2])
                m.mcmc_sweep(sg, st, 2, 4, 1, tr[2:])
            else:
                m.mcmc_sweep(sg, st, 0, 6, 1, tr)
            outs.append((sg.cpu().numpy(), st.cpu().numpy(), tr.cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_fp32_sampler_energy_matches_exact():
    rtt = _rtt()
    inst = inputs.workload("tiny_fp64")
    e_exact = orc.Oracle(inst).exact_energy()
    B, T = 512, 400
    with rtt.RTT(inst, "fp32", seed=99) as m:
        sg = torch.from_numpy(inputs.initial_spins(4, B, 9)).cuda()
        _, _, st = m.log_amplitudes(sg)
        m.mcmc_sweep(sg, st, 0, 100, 1, None)
        tr = torch.empty((T, B), dtype=torch.float64, device="cuda")
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        m.mcmc_sweep(sg, st, 100, T, 1, tr, acc)
        stats = m.observables(tr, acc, T * 9)
    assert abs(stats["mean"] - e_exact) < 3.5 * stats["se"], (stats, e_exact)
    assert 0 < stats["accept_rate"] < 1


def test_observables_match_oracle_statistics():
    rtt = _rtt()
    rng = np.random.default_rng(5)
    T, B = 300, 97
    x = np.empty((T, B))
    x[0] = rng.standard_normal(B)
    for t in range(1, T):
        x[t] = 0.7 * x[t - 1] + rng.standard_normal(B)
    x += -30.0
    acc = rng.integers(0, 1000, B).astype(np.int64)
    ref = orc.observables(x, 36, acc, 2000)
    inst = inputs.workload("tiny_fp64")
    with rtt.RTT(inst, "fp64") as m:
        got = m.observables(torch.from_numpy(x).cuda(), torch.from_numpy(acc).cuda(), 2000)
    for k in ("mean", "var", "tau_int", "ess", "se", "se_bin", "se_chain", "accept_rate"):
        assert got[k] == pytest.approx(ref[k], rel=1e-9), k
    assert got["window"] == ref["window"]
    assert got["v_score"] == pytest.approx(9 * ref["var"] / ref["mean"] ** 2, rel=1e-9)


# ---------------------------------------------------------------- edge cases

def test_empty_and_single_chain():
    rtt = _rtt()
    inst = inputs.workload("tiny_fp64")
    o = orc.Oracle(inst)
    with rtt.RTT(inst, "fp64") as m:
        empty = torch.empty((0, 9), dtype=torch.uint8, device="cuda")
        la, sg, st = m.log_amplitudes(empty)
        assert la.numel() == 0
        e = m.local_energy(empty)
        assert e.numel() == 0
        m.mcmc_sweep(empty, rtt.new_state(0), 0, 3)
        one = inputs.initial_spins(1, 1, 9)
        e1 = m.local_energy(torch.from_numpy(one).cuda()).cpu().numpy()
    assert e1[0] == o.local_energies(one)[0]


def test_argument_errors_raise():
    rtt = _rtt()
    inst = inputs.workload("tiny_fp64")
    with rtt.RTT(inst, "fp32") as m:
        sg = torch.zeros((4, 9), dtype=torch.uint8, device="cuda")
        st = rtt.new_state(4)
        with pytest.raises(rtt.RTTError) as ei:
            m.mcmc_sweep(sg, st, 0, 2, 0, torch.empty((1, 4), dtype=torch.float64, device="cuda"))
        assert ei.value.status == 1


# ---------------------------------------------------------------- full-size workload

def test_plain_6x6_full_batch_sampled_against_oracle():
    """4096 chains of the 6x6 / R=2 / chi=64 workload in FP64 and FP32:
    sampled chains are recomputed by the oracle one by one from the seeded
    start (each picked chain run alone under its own chain index)."""
    rtt = _rtt()
    w = inputs.WORKLOADS["plain_6x6"]
    inst = inputs.workload("plain_6x6")
    o = orc.Oracle(inst)
    B = w["chains"]
    s0 = inputs.initial_spins(w["seed"], B, inst.n_spins)
    pick = np.array([0, 1, 2047, 3000, B - 1])
    # the oracle's own chains: the picked configurations after two sweeps
    so = s0[pick].copy()
    for k, c in enumerate(pick):
        sc = s0[c:c + 1].copy()
        mc, ec = o.init_chains(sc)
        o.mcmc(w["seed"], sc, mc, ec, 0, 2, chain0=int(c), record=False)
        so[k] = sc[0]
    la_o, _, _, _ = o.log_amplitudes(s0[pick])
    e0_o, r0_o = o.local_energies(s0[pick], with_ratios=True, threads=5)
    e2_o, r2_o = o.local_energies(so, with_ratios=True, threads=5)
    # FP32 bound as for the local energy alone: 2e-5 (|J| n_bonds + |h| sum_i |ratio_i|)
    sc0 = abs(inst.J) * inst.bonds.shape[0] + abs(inst.h) * np.abs(r0_o).sum(axis=1)
    sc2 = abs(inst.J) * inst.bonds.shape[0] + abs(inst.h) * np.abs(r2_o).sum(axis=1)
    for prec in ("fp64", "fp32"):
        with rtt.RTT(inst, prec, seed=w["seed"]) as m:
            sg = torch.from_numpy(s0.copy()).cuda()
            la, _, st = m.log_amplitudes(sg)
            tr = torch.empty((2, B), dtype=torch.float64, device="cuda")
            m.mcmc_sweep(sg, st, 0, 1, 1, tr[0:1])
            spins_mid = sg.cpu().numpy()
            m.mcmc_sweep(sg, st, 1, 1, 1, tr[1:2])
            e_now = m.local_energy(sg).cpu().numpy()
            torch.cuda.synchronize()
            spins_now = sg.cpu().numpy()
        la = la.cpu().numpy()
        e_in = tr[0].cpu().numpy()      # the trace measures the configuration entering each sweep
        if prec == "fp64":
            # FP64 chains are bit-exact: the same spins, so the same energies
            assert np.array_equal(spins_now[pick], so)
            assert np.array_equal(la[pick], la_o)
            assert np.array_equal(e_now[pick], e2_o)
            assert np.array_equal(e_in[pick], e0_o)
        else:
            assert np.all(np.abs(la[pick] - la_o) <= fp32_logpsi_tol(o, s0[pick], la_o))
            assert np.all(np.abs(e_in[pick] - e0_o) <= 2e-5 * sc0)
            # both sweeps' decisions replayed by the oracle: every divergence
            # from the FP64 rule an explained near tie
            for a, b, sweep in ((s0, spins_mid, 0), (spins_mid, spins_now, 1)):
                for c in pick:
                    check_sweep_divergences(o, w["seed"], a[c:c + 1], b[c:c + 1], sweep,
                                            eps_site(64, "fp32"), chain0=int(c))
            # the final energies against the oracle on the same configurations
            e3_o, r3_o = o.local_energies(spins_now[pick], with_ratios=True, threads=5)
            sc3 = abs(inst.J) * inst.bonds.shape[0] + abs(inst.h) * np.abs(r3_o).sum(axis=1)
            assert np.all(np.abs(e_now[pick] - e3_o) <= 2e-5 * sc3)
