"""Dual Monte Carlo (Sec. 3.3) on the GPU against the FP64 oracle: mixed local
energies and overlap ratios per configuration, direct sums of RTTs, and the
sampled H~ / S~ matrices and their generalized eigenvalues."""
import numpy as np
import pytest
import torch

from paper_2604_22718_gb300 import inputs
from oracle import oracle as orc
from oracle import dual

pytestmark = pytest.mark.gpu


def _rtt():
    from paper_2604_22718_gb300 import rtt
    return rtt


def _pair(lx, R, chi, seeds, mixing=True, h=3.0):
    return [inputs.make_instance(lx, lx, R, chi, h, seed=s, mixing=mixing) for s in seeds]


@pytest.mark.parametrize("lx,R,chi,B", [(3, 2, 8, 300), (6, 2, 64, 129)])
def test_fp64_mixed_local_energy_bit_exact(lx, R, chi, B):
    rtt = _rtt()
    a, b = _pair(lx, R, chi, (51, 52))
    spins = inputs.initial_spins(53, B, lx * lx)
    e_o, r_o = dual.mixed_local_energies(orc.Oracle(a), orc.Oracle(b), spins, threads=8)
    with rtt.RTT(a, "fp64") as ma, rtt.RTT(b, "fp64") as mb:
        e, r = ma.mixed_local_energy(mb, torch.from_numpy(spins).cuda())
        e_ab, r_aa = ma.mixed_local_energy(ma, torch.from_numpy(spins).cuda())
        e_loc = ma.local_energy(torch.from_numpy(spins).cuda())
        torch.cuda.synchronize()
    assert np.array_equal(e.cpu().numpy(), e_o)
    assert np.array_equal(r.cpu().numpy(), r_o)
    assert np.all(r_aa.cpu().numpy() == 1.0)
    np.testing.assert_allclose(e_ab.cpu().numpy(), e_loc.cpu().numpy(), rtol=1e-13, atol=1e-13)


U32 = 2.0 ** -24
U16 = {"fp16x3": 2.0 ** -11}


def _logpsi_tol(o, spins, prec, chi):
    """Allowed |d log|psi|| per configuration: FP32 as the SIMT tests (1e-5
    relative plus the closing contraction's amplification 2 u32 sqrt(L)
    kappa_fin); split precision by its first-order bound eps_site (sum kappa_k
    + kappa_fin), eps_site = 3 u16^2 + chi u32."""
    cond = o.amplitude_cond(spins)
    if prec == "fp32":
        la = o.log_amplitudes(spins)[0]
        return 1e-5 * np.maximum(1.0, np.abs(la)) + 2 * U32 * np.sqrt(o.L) * cond[:, 2]
    return (3 * U16[prec] ** 2 + chi * U32) * (cond[:, 0] + cond[:, 2])


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_low_precision_mixed_local_energy(prec):
    """Ratio and mixed energy within the error propagated from the amplitudes:
    r = psi^b(s)/psi^a(s) to (tol_a + tol_b) |r|, and E^{ab} to
    |J zz r| (tol_a + tol_b) + h sum_i |r_i| (tol_a + tol_b(s^(i)))."""
    rtt = _rtt()
    a, b = _pair(6, 2, 64, (54, 55))
    B, N = 160, 36
    spins = inputs.initial_spins(56, B, N)
    oa, ob = orc.Oracle(a), orc.Oracle(b)
    e_o, r_o = dual.mixed_local_energies(oa, ob, spins, threads=8)
    with rtt.RTT(a, prec) as ma, rtt.RTT(b, prec) as mb:
        e, r = ma.mixed_local_energy(mb, torch.from_numpy(spins).cuda())
        torch.cuda.synchronize()
    e, r = e.cpu().numpy(), r.cpu().numpy()
    flips = np.repeat(spins, N, axis=0)
    flips[np.arange(B * N), np.tile(np.arange(N), B)] ^= 1
    ta = _logpsi_tol(oa, spins, prec, 64)
    tb = _logpsi_tol(ob, spins, prec, 64)
    tbf = _logpsi_tol(ob, flips, prec, 64).reshape(B, N)
    la_a = oa.log_amplitudes(spins)[0]
    ri = np.exp(ob.log_amplitudes(flips)[0].reshape(B, N) - la_a[:, None])
    zz = np.array([sum((1 - 2 * int(x[i])) * (1 - 2 * int(x[j])) for i, j in a.bonds) for x in spins])
    assert np.all(np.abs(r - r_o) <= 1.01 * (ta + tb) * np.abs(r_o))
    bound = np.abs(a.J * zz * r_o) * (ta + tb) + a.h * np.sum(ri * (ta[:, None] + tbf), axis=1)
    assert np.all(np.abs(e - e_o) <= 1.01 * bound + 1e-12 * np.abs(e_o))
    print(prec, "median rel. ratio error", np.median(np.abs(r - r_o) / np.abs(r_o)))


def test_mixed_energy_rejects_other_lattice():
    rtt = _rtt()
    a = inputs.make_instance(3, 3, 2, 8, 3.0, seed=1)
    b = inputs.make_instance(3, 3, 2, 8, 3.1, seed=2)
    with rtt.RTT(a, "fp64") as ma, rtt.RTT(b, "fp64") as mb:
        with pytest.raises(rtt.RTTError):
            ma.mixed_local_energy(mb, torch.zeros((4, 9), dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_direct_sum_handle_amplitudes(prec):
    rtt = _rtt()
    if prec == "fp64":
        states = _pair(3, 2, 4, (61, 62, 63), mixing=False)
        coef = np.array([0.5, -1.25, 2.0])
    else:
        states = _pair(6, 2, 64, (61, 62))
        coef = np.array([1.0, -0.375])
    s_sum = dual.direct_sum(states, coef)
    o = orc.Oracle(s_sum)
    spins = inputs.initial_spins(64, 257, states[0].n_spins)
    la_o, sg_o, _, _ = o.log_amplitudes(spins)
    with rtt.RTT.from_sum(states, coef, prec) as m, rtt.RTT(s_sum, prec) as m2:
        la, sg, _ = m.log_amplitudes(torch.from_numpy(spins).cuda())
        la2, sg2, _ = m2.log_amplitudes(torch.from_numpy(spins).cuda())
        torch.cuda.synchronize()
    la, sg, la2, sg2 = la.cpu().numpy(), sg.cpu().numpy(), la2.cpu().numpy(), sg2.cpu().numpy()
    assert np.array_equal(la, la2) and np.array_equal(sg, sg2)    # same handle content
    if prec == "fp64":
        assert np.array_equal(la, la_o) and np.array_equal(sg, sg_o)
    else:
        cond = o.amplitude_cond(spins)
        ok = np.abs(la - la_o) <= (3 * 2.0 ** -22 + 128 * 2.0 ** -24) * (cond[:, 0] + cond[:, 2])
        assert ok.mean() > 0.99


def _sample_tilde(rtt, hs, B, T, burn, seed0):
    """Per state a: B chains of P^a on the GPU, after burn sweeps T measured
    sweeps, mixed energies and ratios against every b.  Returns host arrays
    e[a][b][T][B], r[a][b][T][B]."""
    M = len(hs)
    n = hs[0].n
    e_all = np.empty((M, M, T, B))
    r_all = np.empty((M, M, T, B))
    for a_i, ma in enumerate(hs):
        sp = torch.from_numpy(inputs.initial_spins(seed0 + a_i, B, n)).cuda()
        _, _, st = ma.log_amplitudes(sp)
        ma.mcmc_sweep(sp, st, 0, burn)
        e_tr = torch.empty((M, T, B), dtype=torch.float64, device="cuda")
        r_tr = torch.empty((M, T, B), dtype=torch.float64, device="cuda")
        for t in range(T):
            ma.mcmc_sweep(sp, st, burn + t, 1)
            for b_i, mb in enumerate(hs):
                e, r = ma.mixed_local_energy(mb, sp)
                e_tr[b_i, t] = e
                r_tr[b_i, t] = r
        e_all[a_i] = e_tr.cpu().numpy()
        r_all[a_i] = r_tr.cpu().numpy()
    return e_all, r_all


def test_sampled_dual_matrices_against_exact():
    """M = 3 states of a 3x3 lattice: chains of each state sample P^a on the GPU;
    mixed energies and ratios against every b give H~ and S~ within 4.5 SE of
    the enumerated values (SE from rtt_observables); the lowest generalized
    eigenvalue (rtt_dual_solve) is within 4.5 SE of the exact one, its SE from
    the spread over 8 groups of disjoint chains."""
    rtt = _rtt()
    states = _pair(3, 2, 4, (71, 72, 73))
    Ht_x, St_x = dual.exact_tilde_matrices(states)
    M, B, T, burn, G = 3, 2048, 60, 30, 8
    hs = [rtt.RTT(s, "fp64", seed=900 + k) for k, s in enumerate(states)]
    e_all, r_all = _sample_tilde(rtt, hs, B, T, burn, 80)
    Hm, Hse, Sm, Sse = (np.zeros((M, M)) for _ in range(4))
    for a_i in range(M):
        for b_i in range(M):
            se = hs[a_i].observables(torch.from_numpy(e_all[a_i, b_i]).cuda())
            sr = hs[a_i].observables(torch.from_numpy(r_all[a_i, b_i]).cuda())
            Hm[a_i, b_i], Hse[a_i, b_i] = se["mean"], se["se"]
            Sm[a_i, b_i], Sse[a_i, b_i] = sr["mean"], sr["se"]
    for m in hs:
        m.close()
    Hse, Sse = np.nan_to_num(Hse), np.nan_to_num(Sse)     # a constant trace has no error
    assert np.all(np.abs(Hm - Ht_x) <= 4.5 * Hse + 1e-12), (Hm, Ht_x, Hse)
    assert np.all(np.abs(Sm - St_x) <= 4.5 * Sse + 1e-12), (Sm, St_x, Sse)
    assert np.all(np.diag(Sm) == 1.0)
    w, _ = rtt.dual_solve(Hm, Sm)
    w_x, _ = dual.solve(Ht_x, St_x)
    lam_g = []
    for g in range(G):
        sl = slice(g * B // G, (g + 1) * B // G)
        wg, _ = rtt.dual_solve(e_all[:, :, :, sl].mean(axis=(2, 3)), r_all[:, :, :, sl].mean(axis=(2, 3)))
        lam_g.append(wg.real[0])
    se_lam = np.std(lam_g, ddof=1) / np.sqrt(G)
    print("lambda0 sampled", w.real[0], "exact", w_x.real[0], "SE", se_lam)
    assert abs(w.real[0] - w_x.real[0]) <= 4.5 * se_lam, (w, w_x, se_lam)


def test_gram_schmidt_states_on_gpu():
    """Gram-Schmidt against psi^1 (Eq. Gram-Schmid) with exact S~: the new
    states are direct-sum handles (rtt_create_sum); on samples of P^1 their
    ratio to psi^1 averages to zero within 4.5 SE, and the mixed energies of
    psi'^m agree with the oracle bit for bit (FP64)."""
    rtt = _rtt()
    states = _pair(3, 2, 4, (74, 75, 76))
    _, St_x = dual.exact_tilde_matrices(states)
    T_gs = dual.gram_schmidt(St_x, first_only=True)
    base = rtt.RTT(states[0], "fp64", seed=990)
    news = [rtt.RTT.from_sum(states, T_gs[m], "fp64") for m in range(1, 3)]
    B, T, burn = 4096, 40, 30
    sp = torch.from_numpy(inputs.initial_spins(91, B, 9)).cuda()
    _, _, st = base.log_amplitudes(sp)
    base.mcmc_sweep(sp, st, 0, burn)
    for k, mn in enumerate(news):
        r_tr = torch.empty((T, B), dtype=torch.float64, device="cuda")
        for t in range(T):
            base.mcmc_sweep(sp, st, burn + 100 * k + t, 1)
            _, r = base.mixed_local_energy(mn, sp)
            r_tr[t] = r
        sr = base.observables(r_tr)
        assert abs(sr["mean"]) <= 4.5 * sr["se"], sr
        spins = inputs.initial_spins(92 + k, 64, 9)       # seeded, the same on both sides
        e_o, r_o = dual.mixed_local_energies(orc.Oracle(states[0]),
                                             orc.Oracle(dual.direct_sum(states, T_gs[k + 1])), spins)
        e, r = base.mixed_local_energy(mn, torch.from_numpy(spins).cuda())
        assert np.array_equal(e.cpu().numpy(), e_o) and np.array_equal(r.cpu().numpy(), r_o)
    base.close()
    for mn in news:
        mn.close()


@pytest.mark.parametrize("prec,lx,chi", [("fp64", 3, 8), ("fp16x3", 6, 64)])
def test_dual_step_equals_separate_calls(prec, lx, chi):
    """rtt_dual_step (measurements on the second stream beside the sweeps) gives
    bit for bit what rtt_mixed_local_energy on the entering configurations and
    then one rtt_mcmc_sweep per state give on one stream."""
    rtt = _rtt()
    states = _pair(lx, 2, chi, (81, 82, 83))
    M, B, n = 3, 300, lx * lx
    hs = [rtt.RTT(s, prec, seed=700 + k) for k, s in enumerate(states)]
    sp0 = [torch.from_numpy(inputs.initial_spins(110 + k, B, n)).cuda() for k in range(M)]
    st0 = [h.log_amplitudes(x)[2] for h, x in zip(hs, sp0)]
    # separate calls
    sp1 = [x.clone() for x in sp0]
    st1 = [x.clone() for x in st0]
    e1 = torch.empty((M, M, B), dtype=torch.float64, device="cuda")
    r1 = torch.empty((M, M, B), dtype=torch.float64, device="cuda")
    acc1 = [torch.zeros(B, dtype=torch.int64, device="cuda") for _ in range(M)]
    for a in range(M):
        for b in range(M):
            e, r = hs[a].mixed_local_energy(hs[b], sp1[a])
            e1[a, b], r1[a, b] = e, r
        hs[a].mcmc_sweep(sp1[a], st1[a], 5, 1, n_accept=acc1[a])
    # one dual step
    sp2 = [x.clone() for x in sp0]
    st2 = [x.clone() for x in st0]
    e2 = torch.empty((M, M, B), dtype=torch.float64, device="cuda")
    r2 = torch.empty((M, M, B), dtype=torch.float64, device="cuda")
    acc2 = [torch.zeros(B, dtype=torch.int64, device="cuda") for _ in range(M)]
    rtt.dual_step(hs, sp2, st2, 5, e2, r2, acc2)
    torch.cuda.synchronize()
    assert torch.equal(e1, e2) and torch.equal(r1, r2)
    for a in range(M):
        assert torch.equal(sp1[a], sp2[a]) and torch.equal(st1[a], st2[a])
        assert torch.equal(acc1[a], acc2[a])
    for h in hs:
        h.close()
