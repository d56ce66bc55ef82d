"""GPU parity of the tensor-core split-precision paths (tcgen05; BF16 and FP16
hi/lo operands) against the FP64 oracle, through the C ABI.

Split-precision bound (first order): with 16-bit unit roundoff u_b (BF16
2^-8, FP16 2^-11) the split x = hi + lo leaves |x - hi - lo| <= u_b^2 |x|,
and the dropped lo.lo product is <= u_b^2 |x||y|; FP32 accumulation of chi
terms adds chi u_32.  So
every site product carries a componentwise error <= eps_site (|v||A|)_b with
eps_site = 3 u_b^2 + chi u_32, i.e. a relative error <= eps_site kappa_k in
norm, and the closing contraction <= eps_site kappa_fin.  Hence
|d log|psi|| <= eps_site (sum_k kappa_k + kappa_fin), with the kappas computed
per configuration by the oracle in FP64."""

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2604_22718_gb300 import inputs
from parity_util import check_sweep_divergences, local_energy_bound

pytestmark = pytest.mark.gpu

UB = {"bf16x3": 2.0 ** -8, "fp16x3": 2.0 ** -11}
U32 = 2.0 ** -24
PRECS = ["bf16x3", "fp16x3"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2604_22718_gb300 import build
    build.build()


def _rtt():
    from paper_2604_22718_gb300 import rtt
    return rtt


def eps_site(chi, prec):
    return 3 * UB[prec] ** 2 + chi * U32


def _status_ok(m):
    rtt = _rtt()
    flags = rtt.ctypes.c_int32()
    st = rtt.lib().rtt_device_status(m.handle, rtt.ctypes.byref(flags))
    return st == 0 and flags.value == 0


@pytest.mark.parametrize("prec", PRECS)
def test_first_light_tiny_train_matches_fp32(prec):
    """Smallest case first: one partial tile, L = 8 sites, chi = 64."""
    rtt = _rtt()
    inst = inputs.make_instance(2, 2, 2, 64, 3.0, seed=31)
    spins = torch.from_numpy(inputs.initial_spins(31, 37, 4)).cuda()
    with rtt.RTT(inst, "fp32") as m32:
        la32, sg32, _ = m32.log_amplitudes(spins)
    with rtt.RTT(inst, prec) as mtc:
        la, sg, _ = mtc.log_amplitudes(spins)
        torch.cuda.synchronize()
        assert _status_ok(mtc)
    la, la32 = la.cpu().numpy(), la32.cpu().numpy()
    print("first light: max |dlog| vs fp32", np.max(np.abs(la - la32)))
    assert np.all(np.isfinite(la))
    assert np.max(np.abs(la - la32)) < 1e-2
    assert np.array_equal(sg.cpu().numpy(), sg32.cpu().numpy())


CASES = [
    ("6x6_R2_chi64", lambda: inputs.make_instance(6, 6, 2, 64, 3.0, seed=5), 300),
    ("3x3_R2_chi64", lambda: inputs.make_instance(3, 3, 2, 64, 3.0, seed=8), 129),
    ("4x5_R3_chi128", lambda: inputs.make_instance(4, 5, 3, 128, 3.04, seed=9), 200),
    ("3x4_R1_chi128_mps", lambda: inputs.make_instance(3, 4, 1, 128, 3.0, seed=10), 64),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,make,B", CASES, ids=[c[0] for c in CASES])
def test_split_log_amplitudes_within_bound(name, make, B, prec):
    rtt = _rtt()
    inst = make()
    o = orc.Oracle(inst)
    spins = inputs.initial_spins(41, B, inst.n_spins)
    la_o, sg_o, _, _ = o.log_amplitudes(spins)
    cond = o.amplitude_cond(spins)
    with rtt.RTT(inst, prec) as m:
        la, sg, _ = m.log_amplitudes(torch.from_numpy(spins).cuda())
        torch.cuda.synchronize()
        assert _status_ok(m)
    la, sg = la.cpu().numpy(), sg.cpu().numpy()
    err = np.abs(la - la_o)
    bound = eps_site(inst.chi, prec) * (cond[:, 0] + cond[:, 2])
    print(f"[{name}] {prec} log|psi|: median err {np.median(err):.2e}, max {err.max():.2e}, "
          f"max err/bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)
    ok_sign = (sg == sg_o) | (cond[:, 2] * eps_site(inst.chi, prec) > 0.5)
    assert np.all(ok_sign)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,make,B", CASES, ids=[c[0] for c in CASES])
def test_split_local_energy_teacher_forced(name, make, B, prec):
    """Same configurations through the FP64 oracle and the split path.  Every
    ratio psi(s^(i))/psi(s) obeys the split bound of its two amplitudes,
    |dr| <= |r| eps_site (K(s) + K(s^(i))), K = sum_k kappa_k + kappa_fin from
    the oracle, and so every local energy the bound that follows from them.
    FP16X3 also meets the precision gate of the metric (the mean local energy
    within 1e-4 relative, of the mean |E_loc| when the mean is near zero)
    wherever that bound itself lies within the gate: the R = 1 case with
    random chi = 128 cores has ratios large enough that it does not."""
    rtt = _rtt()
    inst = make()
    o = orc.Oracle(inst)
    B = min(B, 48)
    spins = inputs.initial_spins(42, B, inst.n_spins)
    e_o, r_o = o.local_energies(spins, with_ratios=True, threads=16)
    with rtt.RTT(inst, prec) as m:
        e, r = m.local_energy(torch.from_numpy(spins).cuda(), with_ratios=True)
        torch.cuda.synchronize()
        assert _status_ok(m)
    e, r = e.cpu().numpy(), r.cpu().numpy()
    eps = eps_site(inst.chi, prec)
    K = o.amplitude_cond(spins)
    K = K[:, 0] + K[:, 2]
    nc = min(B, 12)
    flipped = np.repeat(spins[:nc], inst.n_spins, axis=0)
    idx = np.tile(np.arange(inst.n_spins), nc)
    flipped[np.arange(flipped.shape[0]), idx] ^= 1
    Kf = o.amplitude_cond(flipped)
    Kf = (Kf[:, 0] + Kf[:, 2]).reshape(nc, inst.n_spins)
    bound = np.abs(r_o[:nc]) * eps * (K[:nc, None] + Kf)
    dr = np.abs(r[:nc] - r_o[:nc])
    de = abs(e.mean() - e_o.mean())
    rel_mean = de / max(abs(e_o.mean()), np.mean(np.abs(e_o)))
    print(f"[{name}] {prec} E_loc: mean rel err {rel_mean:.2e} (|dE| {de:.2e}), "
          f"max |dr|/bound {np.max(dr / bound):.3f}, median |dr|/|r| {np.median(dr / np.abs(r_o[:nc])):.2e}")
    assert np.all(dr <= bound)
    ebound = local_energy_bound(o, spins, r_o, eps, inst.J, inst.h, inst.bonds.shape[0])
    scale = max(abs(e_o.mean()), np.mean(np.abs(e_o)))
    print(f"[{name}] {prec} E_loc: max |dE|/bound {np.max(np.abs(e - e_o) / ebound):.3f}, "
          f"mean bound / scale {ebound.mean() / scale:.2e}")
    assert np.all(np.abs(e - e_o) <= ebound)
    assert de <= ebound.mean()
    if prec == "fp16x3" and ebound.mean() <= 1e-4 * scale:
        assert rel_mean <= 1e-4


@pytest.mark.parametrize("prec", PRECS)
def test_split_sampler_energy_matches_exact(prec):
    rtt = _rtt()
    inst = inputs.make_instance(3, 3, 2, 64, 3.0, seed=8)
    e_exact = orc.Oracle(inst).exact_energy()
    B, T = 512, 300
    with rtt.RTT(inst, prec, seed=7) as m:
        sg = torch.from_numpy(inputs.initial_spins(43, B, 9)).cuda()
        _, _, st = m.log_amplitudes(sg)
        m.mcmc_sweep(sg, st, 0, 60, 1, None)
        tr = torch.empty((T, B), dtype=torch.float64, device="cuda")
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        m.mcmc_sweep(sg, st, 60, T, 1, tr, acc)
        stats = m.observables(tr, acc, T * 9)
        assert _status_ok(m)
    print(prec, "sampler", stats, "exact", e_exact)
    assert abs(stats["mean"] - e_exact) < 3.5 * stats["se"], (stats, e_exact)
    assert 0 < stats["accept_rate"] < 1


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("R,chi", [(2, 64), (2, 128), (1, 128)])
def test_split_sweep_follows_oracle_decisions(prec, R, chi):
    """One sweep from the same start: every decision the split-precision sweep
    takes is the FP64 rule's at the same state, except at near ties |u - r^2|
    within the ratio bound; none is left unexplained.  R = 2 runs the
    split-row sweeps on CTA pairs, R = 1 the single-tile sweep."""
    rtt = _rtt()
    inst = inputs.make_instance(6, 6, R, chi, 3.0, seed=5)
    o = orc.Oracle(inst)
    B = 64
    s0 = inputs.initial_spins(44, B, 36)
    with rtt.RTT(inst, prec, seed=11) as m:
        sg = torch.from_numpy(s0.copy()).cuda()
        _, _, st = m.log_amplitudes(sg)
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        m.mcmc_sweep(sg, st, 0, 1, 1, None, acc)
        torch.cuda.synchronize()
        assert _status_ok(m)
    s1 = sg.cpu().numpy()
    n, nd, worst = check_sweep_divergences(o, 11, s0, s1, 0, eps_site(chi, prec),
                                           slack=2.0 ** -23)
    print(prec, chi, f"sweep: {nd} of {n} decisions differ from FP64, all near ties "
                     f"(largest gap / tolerance {worst:.3f})")
    assert np.array_equal(acc.cpu().numpy(),
                          np.sum(s1[:, inst.path[:36]] != s0[:, inst.path[:36]], axis=1))


@pytest.mark.parametrize("chi", [64, 128])
def test_split_two_sweeps_in_one_call_equal_two_calls(chi):
    """Two sweeps in one call (the sweep boundary inside the kernel: the right
    environment rebuilt from the new spins, the left row restarted from b_L)
    give the same spins, amplitudes and acceptance counts, bit for bit, as two
    calls of one sweep each; each of those sweeps follows the FP64 rule except
    at explained near ties.  Two tiles, the second ragged."""
    rtt = _rtt()
    inst = inputs.make_instance(6, 6, 2, chi, 3.0, seed=5)
    o = orc.Oracle(inst)
    B = 200
    s0 = inputs.initial_spins(46, B, 36)
    with rtt.RTT(inst, "fp16x3", seed=13) as m:
        sa_ = torch.from_numpy(s0.copy()).cuda()
        _, _, sta = m.log_amplitudes(sa_)
        sb = sa_.clone()
        stb = sta.clone()
        acca = torch.zeros(B, dtype=torch.int64, device="cuda")
        accb = torch.zeros(B, dtype=torch.int64, device="cuda")
        m.mcmc_sweep(sa_, sta, 0, 2, 1, None, acca)
        m.mcmc_sweep(sb, stb, 0, 1, 1, None, accb)
        s_mid = sb.cpu().numpy()
        m.mcmc_sweep(sb, stb, 1, 1, 1, None, accb)
        torch.cuda.synchronize()
        assert _status_ok(m)
    assert torch.equal(sa_, sb) and torch.equal(sta, stb) and torch.equal(acca, accb)
    eps = eps_site(chi, "fp16x3")
    for sw, (x0, x1) in enumerate([(s0, s_mid), (s_mid, sb.cpu().numpy())]):
        n, nd, worst = check_sweep_divergences(o, 13, x0, x1, sw, eps, slack=2.0 ** -23)
        print(chi, f"sweep {sw}: {nd} of {n} decisions differ from FP64 (worst {worst:.3f})")


@pytest.mark.parametrize("prec", PRECS)
def test_split_measured_trace_equals_standalone_energy(prec):
    rtt = _rtt()
    inst = inputs.make_instance(4, 5, 3, 128, 3.04, seed=9)
    B = 200
    with rtt.RTT(inst, prec, seed=3) as m:
        sg = torch.from_numpy(inputs.initial_spins(45, B, 20)).cuda()
        _, _, st = m.log_amplitudes(sg)
        e0 = m.local_energy(sg)
        tr = torch.empty((2, B), dtype=torch.float64, device="cuda")
        m.mcmc_sweep(sg, st, 0, 2, 1, tr)      # measures the states entering sweeps 0 and 1
        e2 = m.local_energy(sg)
        tr2 = torch.empty((1, B), dtype=torch.float64, device="cuda")
        m.mcmc_sweep(sg, st, 2, 1, 1, tr2)
        torch.cuda.synchronize()
        assert _status_ok(m)
    # the measurement beside the sweep runs the standalone kernels on a snapshot
    assert np.array_equal(tr[0].cpu().numpy(), e0.cpu().numpy())
    assert np.array_equal(tr2[0].cpu().numpy(), e2.cpu().numpy())
    assert not np.array_equal(tr[1].cpu().numpy(), tr[0].cpu().numpy())


@pytest.mark.parametrize("prec", PRECS)
def test_prec_10x10_full_batch_sampled_against_oracle(prec):
    """The 10x10 / R=3 / chi=128 workload at its full 16384 chains: amplitudes
    and local energies of picked chains against the oracle one by one, each
    within its own split bound, and the decisions of one full-batch sweep of
    the picked chains, every divergence a near tie."""
    rtt = _rtt()
    w = inputs.WORKLOADS["prec_10x10"]
    inst = inputs.workload("prec_10x10")
    o = orc.Oracle(inst)
    B = w["chains"]
    s0 = inputs.initial_spins(w["seed"], B, inst.n_spins)
    pick = np.array([0, 5000, B - 1])
    with rtt.RTT(inst, prec, seed=w["seed"]) as m:
        sg = torch.from_numpy(s0.copy()).cuda()
        la, _, st = m.log_amplitudes(sg)
        e, r = m.local_energy(sg, with_ratios=True)
        tr = torch.empty((1, B), dtype=torch.float64, device="cuda")
        m.mcmc_sweep(sg, st, 0, 1, 1, tr)
        torch.cuda.synchronize()
        assert _status_ok(m)
        s1 = sg.cpu().numpy()
    la, e, r = la.cpu().numpy(), e.cpu().numpy(), r.cpu().numpy()
    eps = eps_site(128, prec)
    la_o, _, _, _ = o.log_amplitudes(s0[pick])
    cond = o.amplitude_cond(s0[pick])
    assert np.all(np.abs(la[pick] - la_o) <= eps * (cond[:, 0] + cond[:, 2]))
    e_o, r_o = o.local_energies(s0[pick], with_ratios=True, threads=3)
    bound = local_energy_bound(o, s0[pick], r_o, eps, inst.J, inst.h, inst.bonds.shape[0])
    print("prec_10x10 E_loc sampled", e[pick], e_o, "bound", bound)
    assert np.all(np.abs(e[pick] - e_o) <= bound)
    assert np.array_equal(tr[0].cpu().numpy(), e)        # the trace measures the entering state
    for c in pick:                                       # each under its own chain index
        check_sweep_divergences(o, w["seed"], s0[c:c + 1], s1[c:c + 1], 0, eps, chain0=int(c))


@pytest.mark.parametrize("prec", ["fp16x3"])
def test_learned_16x16_full_batch_sweep_against_oracle(prec):
    """The learned-proposal workload's shape (16x16, R = 2, L = 512, chi =
    128) at its full 8192 chains: one sweep's decisions of picked chains
    (every divergence a near tie), the amplitude each chain tracks against the
    oracle's amplitude of its new spins, and the measured local energies of the
    entering configurations within their split bounds."""
    rtt = _rtt()
    w = inputs.WORKLOADS["learned_16x16"]
    inst = inputs.workload("learned_16x16")
    o = orc.Oracle(inst)
    B = w["chains"]
    N = inst.n_spins
    s0 = inputs.initial_spins(w["seed"], B, N)
    pick = np.array([0, 4097, B - 1])
    with rtt.RTT(inst, prec, seed=w["seed"]) as m:
        sg = torch.from_numpy(s0.copy()).cuda()
        _, _, st = m.log_amplitudes(sg)
        tr = torch.empty((1, B), dtype=torch.float64, device="cuda")
        m.mcmc_sweep(sg, st, 0, 1, 1, tr)
        torch.cuda.synchronize()
        assert _status_ok(m)
        s1 = sg.cpu().numpy()
        la_track = (rtt.state_exp(st).double() * np.log(2.0) +
                    torch.log(rtt.state_mant(st).abs())).cpu().numpy()
    eps = eps_site(128, prec)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(len(pick)) as ex:
        res = list(ex.map(lambda c: check_sweep_divergences(
            o, w["seed"], s0[c:c + 1], s1[c:c + 1], 0, eps, chain0=int(c), threads=1), pick))
    print("learned_16x16 sweep (proposals, divergences, worst):", res)
    la_o, _, _, _ = o.log_amplitudes(s1[pick])
    K = o.amplitude_cond(s1[pick])
    # the tracked amplitude came from the accepted proposals' rows: within the
    # bound of both evaluations
    assert np.all(np.abs(la_track[pick] - la_o) <= 2 * eps * (K[:, 0] + K[:, 2]))
    e_o, r_o = o.local_energies(s0[pick[:2]], with_ratios=True, threads=2)
    bound = local_energy_bound(o, s0[pick[:2]], r_o, eps, inst.J, inst.h, inst.bonds.shape[0])
    e = tr[0].cpu().numpy()[pick[:2]]
    print("learned_16x16 E_loc", e, e_o, "bound", bound)
    assert np.all(np.abs(e - e_o) <= bound)
