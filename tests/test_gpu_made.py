"""Learned independence proposal on the GPU against the FP64 oracle of
oracle/made.py: forward log-probabilities, gradients, Adam, the sampler
(same Philox stream), exact self-consistency of the sampled log q, and the
gain of the trained proposal over local flips on a slowly mixing state."""
import itertools

import numpy as np
import pytest
import torch

from oracle import made
from oracle import oracle as orc
from paper_2604_22718_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2604_22718_gb300 import build
    build.build()


def _rtt():
    from paper_2604_22718_gb300 import rtt
    return rtt


def _setup(N, H, seed=1):
    w = inputs.made_init_weights(seed, N, H)
    # nonzero biases so that they are exercised
    rng = np.random.default_rng(seed)
    o = 0
    for name, shp in made.shapes(N, H):
        n = int(np.prod(shp))
        if name.startswith("b"):
            w[o:o + n] = rng.standard_normal(n) * 0.3
        o += n
    order = np.random.default_rng(seed + 1).permutation(N).astype(np.int32)
    return w, order


def test_log_prob_matches_oracle():
    rtt = _rtt()
    N, H, B = 20, 48, 300
    w, order = _setup(N, H)
    p = made.masked_params(w, N, H)
    spins = inputs.initial_spins(3, B, N)
    with rtt.MADE(N, H, order, w) as m:
        lq = m.log_prob(torch.from_numpy(spins).cuda()).cpu().numpy()
        prm = m.params()
    np.testing.assert_allclose(prm, made.pack(p, N, H), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(lq, made.log_prob(p, spins, order), rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("N,H,B,tc", [(16, 40, 256, False), (16, 40, 256, True), (64, 192, 300, True)])
def test_gradients_match_oracle(N, H, B, tc):
    """Gradients of the NLL against the FP64 oracle, per parameter block within
    1e-4 of its norm: FP32 GEMMs on the CUDA cores, and the tensor-core GEMMs
    (BF16 hi/lo, three products: O(2^-16) per product) on one ragged tile and
    on several tiles with ragged edges in every dimension."""
    rtt = _rtt()
    w, order = _setup(N, H, seed=2)
    p = made.masked_params(w, N, H)
    spins = inputs.initial_spins(4, B, N)
    nll_o, g_o = made.nll_and_grads(p, spins, order, N, H)
    with rtt.MADE(N, H, order, w) as m:
        m.set_training(tc)
        g, nll = m.gradients(torch.from_numpy(spins).cuda())
        g = g.cpu().numpy().astype(np.float64)
        assert m.device_status() == 0
    assert float(nll.cpu()[0]) == pytest.approx(nll_o, rel=1e-6 if not tc else 1e-5)
    go = made.pack(g_o, N, H)
    o = 0
    for name, shp in made.shapes(N, H):
        n = int(np.prod(shp))
        a, b = g[o:o + n], go[o:o + n]
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-9, name
        o += n
    # masked entries stay exactly zero
    assert np.all(g[made.pack(made.apply_masks({k: np.ones(s) for k, s in made.shapes(N, H)}, N, H), N, H) == 0] == 0)


def test_adam_steps_match_oracle():
    rtt = _rtt()
    N, H, B = 12, 32, 128
    w, order = _setup(N, H, seed=3)
    p = made.masked_params(w, N, H)
    mo = {k: np.zeros_like(v) for k, v in p.items()}
    vo = {k: np.zeros_like(v) for k, v in p.items()}
    batches = [inputs.initial_spins(10 + t, B, N) for t in range(3)]
    with rtt.MADE(N, H, order, w) as m:
        # FP32 GEMMs: Adam's first steps move each parameter by about lr times
        # the sign of its gradient, so a near-zero gradient must keep its sign
        m.set_training(False)
        for t, sp in enumerate(batches, start=1):
            _, g = made.nll_and_grads(p, sp, order, N, H)
            p, mo, vo = made.adam_step(p, g, mo, vo, t, lr=1e-2)
            m.train_step(torch.from_numpy(sp).cuda(), lr=1e-2)
        prm = m.params().astype(np.float64)
    np.testing.assert_allclose(prm, made.pack(p, N, H), rtol=2e-4, atol=2e-6)


def test_sampler_matches_oracle_and_reports_its_own_log_prob():
    rtt = _rtt()
    N, H, B = 10, 24, 512
    w, order = _setup(N, H, seed=5)
    p = made.masked_params(w, N, H)
    with rtt.MADE(N, H, order, w, seed=77) as m:
        sp, lq = m.sample(B, chain0=100, round=9)
        lq_fwd = m.log_prob(sp)
        sp, lq, lq_fwd = sp.cpu().numpy(), lq.cpu().numpy(), lq_fwd.cpu().numpy()
    # the density the proposal was drawn from is exactly the one evaluated later
    assert np.array_equal(lq, lq_fwd)
    so, lqo = made.sample(p, order, B, seed=77, chain0=100, rnd=9, N=N)
    same = check_sample_divergences(p, order, sp, so, 77, 100, 9)
    np.testing.assert_allclose(lq[same], lqo[same], rtol=1e-5, atol=1e-5)


def test_sampler_distribution_chi2():
    scipy_stats = pytest.importorskip("scipy.stats")
    rtt = _rtt()
    N, H, B = 8, 16, 40000
    w, order = _setup(N, H, seed=6)
    p = made.masked_params(w, N, H)
    with rtt.MADE(N, H, order, w, seed=5) as m:
        sp, _ = m.sample(B)
        sp = sp.cpu().numpy()
    allc = np.array(list(itertools.product([0, 1], repeat=N)), dtype=np.uint8)
    q = np.exp(made.log_prob(p, allc, order))
    idx = (sp.astype(np.int64) * (1 << np.arange(N - 1, -1, -1))).sum(axis=1)
    obs = np.bincount(idx, minlength=1 << N).astype(float)
    keep = q * B >= 5
    o_b, e_b = obs[keep], q[keep] * B
    if np.any(~keep):
        o_b, e_b = np.append(o_b, obs[~keep].sum()), np.append(e_b, q[~keep].sum() * B)
    e_b *= o_b.sum() / e_b.sum()
    assert scipy_stats.chisquare(o_b, e_b)[1] > 1e-3


def _run_sampler(rtt, m_rtt, made_m, B, T, burn, seed):
    sp = torch.from_numpy(inputs.initial_spins(seed, B, m_rtt.n)).cuda()
    _, _, st = m_rtt.log_amplitudes(sp)
    tr = torch.empty((T, B), dtype=torch.float64, device="cuda")
    acc_i = torch.zeros(B, dtype=torch.int64, device="cuda")
    for t in range(burn + T):
        m_rtt.mcmc_sweep(sp, st, t, 1, 1, tr[max(t - burn, 0):max(t - burn, 0) + 1] if t >= burn else
                         torch.empty((1, B), dtype=torch.float64, device="cuda"))
        if made_m is not None:
            rtt.indep_mh(m_rtt, made_m, sp, st, t, acc_i if t >= burn else None)
    return tr, acc_i, sp


def test_learned_proposal_beats_local_flips_on_a_slowly_mixing_state():
    """A ferromagnetic chain state with a weak field (kappa = 1.3, field 0.05)
    has two polarised modes of unequal weight and local flips almost never
    cross between them: local chains keep the mode populations of their
    start.  A MADE trained on the local sampler's own configurations proposes
    whole configurations; mixed 1:1 with local sweeps it moves chains between
    the modes, reproduces the exact energy and cuts tau_int of E_loc."""
    rtt = _rtt()
    inst = inputs.ferro_chain_instance(3, 4, kappa=1.3, field=0.05, h=1.0)
    N = inst.n_spins
    e_exact = orc.Oracle(inst).exact_energy()
    order = inst.path[:N].astype(np.int32)
    with rtt.RTT(inst, "fp32", seed=3) as m:
        # training data: the local sampler's configurations (many chains, thinned)
        Bd = 4096
        sp = torch.from_numpy(inputs.initial_spins(8, Bd, N)).cuda()
        _, _, st = m.log_amplitudes(sp)
        m.mcmc_sweep(sp, st, 0, 200)
        data = [sp.clone()]
        for r in range(7):
            m.mcmc_sweep(sp, st, 200 + 20 * r, 20)
            data.append(sp.clone())
        data = torch.cat(data)
        with rtt.MADE(N, 64, order, inputs.made_init_weights(4, N, 64), seed=9) as mm:
            hist = mm.fit(data, epochs=15, batch=512, lr=3e-3)
            print("MADE NLL per epoch", [round(h, 4) for h in hist])
            assert hist[-1] < hist[0]
            B, T = 1024, 400
            tr_l, _, _ = _run_sampler(rtt, m, None, B, T, 50, 21)
            tr_m, acc_i, _ = _run_sampler(rtt, m, mm, B, T, 50, 21)
            s_l = m.observables(tr_l)
            s_m = m.observables(tr_m)
    acc_rate = float(acc_i.sum()) / (B * T)
    print("local", s_l, "\nmixed", s_m, "\nexact", e_exact, "indep acceptance", acc_rate)
    assert abs(s_m["mean"] - e_exact) < 3.5 * s_m["se"]
    assert acc_rate > 0.3
    # local flips: populations frozen at their start -- biased or slowly mixing
    assert (abs(s_l["mean"] - e_exact) > 3.5 * s_l["se"]) or (s_m["tau_int"] < 0.5 * s_l["tau_int"])


# ---------------------------------------------------------------- BF16 tensor-core inference

def _bf16_bound(p, spins, order, K):
    """Per configuration, a bound on |log q_bf16 - log q|: the H x H layer's
    products h1_k W2_nk carry at most 2u + u^2 (u = 2^-9, both factors rounded
    to BF16) plus K 2^-24 (FP32 accumulation) of |h1_k W2_nk|; ReLU and
    log-sigmoid are 1-Lipschitz, so the logit error is at most
    sum_n |W3_dn| |da2_n| and the log q error at most the sum over positions.
    A 1e-4 per position allowance covers the FP32 arithmetic of the other
    layers (the FP32 path meets the oracle to 1e-5)."""
    x, _ = made.inputs_of(spins, order)
    a1, h1, a2, h2, lg = made.forward(p, x)
    u = 2.0 ** -9
    rel = 2 * u + u * u + K * 2.0 ** -24
    da2 = rel * (np.abs(h1) @ np.abs(p["W2"]).T)
    dlg = da2 @ np.abs(p["W3"]).T
    return dlg.sum(axis=1) + 1e-4 * x.shape[1]


@pytest.mark.parametrize("N,H", [(16, 64), (9, 128), (11, 192), (12, 256), (10, 512)])
def test_bf16_sampler_reports_its_own_log_prob_and_meets_the_bound(N, H):
    """Tensor-core inference: the sampler's log q is bit for bit the
    evaluation's (same kernel on identical BF16 inputs), and the evaluation
    stays within the BF16 bound of the FP64 oracle's log q on seeded
    configurations."""
    rtt = _rtt()
    B = 1000
    w, order = _setup(N, H, seed=N + H)
    p = made.masked_params(w, N, H)
    seeded = inputs.initial_spins(N + H, B, N)          # the oracle's configurations
    with rtt.MADE(N, H, order, w, seed=41) as m:
        sp, lq = m.sample(B, chain0=3, round=2)
        lq_fwd = m.log_prob(sp)
        lq_s = m.log_prob(torch.from_numpy(seeded).cuda())
        assert m.device_status() == 0
        lq, lq_fwd, lq_s = lq.cpu().numpy(), lq_fwd.cpu().numpy(), lq_s.cpu().numpy()
        m.set_inference(False)
        lq32 = m.log_prob(torch.from_numpy(seeded).cuda()).cpu().numpy()
    assert np.array_equal(lq, lq_fwd)
    ref = made.log_prob(p, seeded, order)
    bound = _bf16_bound(p, seeded, order, H)
    assert np.all(np.abs(lq_s - ref) <= bound), float(np.max(np.abs(lq_s - ref) - bound))
    np.testing.assert_allclose(lq32, ref, rtol=1e-5, atol=1e-5)
    # the bound is not vacuous: BF16 differs from FP32, by less than the bound
    assert np.any(lq_s != lq32)


def test_bf16_needs_a_supported_hidden_width():
    rtt = _rtt()
    N, H = 8, 24
    w, order = _setup(N, H)
    with rtt.MADE(N, H, order, w) as m:
        with pytest.raises(rtt.RTTError, match="UNSUPPORTED"):
            m.set_inference(True)
        m.set_inference(False)


def test_bf16_sampler_distribution_chi2():
    """Samples of the BF16 sampler against its own exact density: the
    evaluation kernel's q over all 2^N configurations (N = 10, H = 64)."""
    rtt = _rtt()
    N, H, B = 10, 64, 1 << 16
    w, order = _setup(N, H, seed=3)
    allc = ((np.arange(1 << N)[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1).astype(np.uint8)
    with rtt.MADE(N, H, order, w, seed=5) as m:
        sp, _ = m.sample(B)
        q = np.exp(m.log_prob(torch.from_numpy(allc).cuda()).cpu().numpy())
        sp = sp.cpu().numpy()
    assert abs(q.sum() - 1.0) < 1e-5
    idx = (sp.astype(np.int64) * (1 << (N - 1 - np.arange(N)))[None, :]).sum(axis=1)
    obs = np.bincount(idx, minlength=1 << N).astype(np.float64)
    exp_ = q * B
    keep = exp_ >= 5
    o, e = obs[keep], exp_[keep]
    if np.any(~keep):                      # bins with few expected counts merged into one
        o, e = np.append(o, obs[~keep].sum()), np.append(e, exp_[~keep].sum())
    chi2 = float(np.sum((o - e) ** 2 / e))
    from scipy.stats import chi2 as c2
    assert c2.sf(chi2, len(o) - 1) > 1e-3


def test_training_loop_equals_train_steps_on_its_row_order():
    """rtt_made_fit gathers each minibatch on the device in the order of
    rtt_made_permutation and takes one Adam step per minibatch: the same steps
    taken one by one on the same rows give bit-identical parameters and the
    same per-epoch mean NLL."""
    rtt = _rtt()
    N, H, n, batch, epochs = 12, 32, 300, 64, 3
    w, order = _setup(N, H, seed=13)
    data = torch.from_numpy(inputs.initial_spins(17, n, N)).cuda()
    with rtt.MADE(N, H, order, w) as a, rtt.MADE(N, H, order, w) as b:
        hist = a.fit(data, epochs=epochs, batch=batch, lr=1e-2, seed=5)
        nll = torch.zeros(1, dtype=torch.float64, device="cuda")
        ref = []
        for e in range(epochs):
            perm = torch.from_numpy(rtt.made_permutation(n, 5, e)).cuda()
            tot = 0.0
            for s in range(0, n - batch + 1, batch):
                b.train_step(data[perm[s:s + batch]].contiguous(), 1e-2, nll)
                tot += float(nll.cpu()[0])
            ref.append(tot / (n // batch))
        pa, pb = a.params(), b.params()
    assert np.array_equal(pa, pb)
    np.testing.assert_allclose(hist, ref, rtol=1e-12)
    assert hist[-1] < hist[0]


# ---------------------------------------------------------------- FP32 bounds
U32 = 2.0 ** -24


def fp32_logit_bound(p, x):
    """Per row and position, a bound on |logit_FP32 - logit| of the forward
    pass on inputs x (+-1): every layer's output adds at most (K + 1) u_32 of
    its absolute sum (K terms accumulated by fma from the bias), ReLU is
    1-Lipschitz, and each layer propagates the error of its input through
    |W|."""
    a1 = np.abs(x) @ np.abs(p["W1"]).T + np.abs(p["b1"])
    d1 = (x.shape[1] + 1) * U32 * a1
    _, h1, _, h2, _ = made.forward(p, x)
    d2 = d1 @ np.abs(p["W2"]).T + (h1.shape[1] + 1) * U32 * (np.abs(h1) @ np.abs(p["W2"]).T + np.abs(p["b2"]))
    return d2 @ np.abs(p["W3"]).T + (h2.shape[1] + 1) * U32 * (np.abs(h2) @ np.abs(p["W3"]).T + np.abs(p["b3"]))


def check_sample_divergences(p, order, sp_gpu, sp_oracle, seed, chain0, rnd):
    """Ancestral samples drawn from the same Philox stream: where a GPU sample
    differs from the oracle's, the first position d at which they differ must
    be a near tie, |u_d - q_d| within the FP32 bound of q_d = sigmoid(logit_d)
    at the common prefix (sigmoid' <= 1/4).  Returns the rows that agree."""
    N = sp_gpu.shape[1]
    same = np.all(sp_gpu == sp_oracle, axis=1)
    for c in np.flatnonzero(~same):
        d = int(np.argmax(sp_gpu[c, order] != sp_oracle[c, order]))
        x = np.zeros((1, N))
        x[0, :d] = 1.0 - 2.0 * sp_oracle[c, order[:d]]
        logit = made.forward(p, x)[4][0, d]
        q = 1.0 / (1.0 + np.exp(-logit))
        u = orc.uniform_keyed(seed, made.MADE_STREAM, chain0 + c, rnd, d)
        tol = fp32_logit_bound(p, x)[0, d] / 4.0 + 1e-12
        assert abs(u - q) <= tol, (c, d, u, q, tol)
    return same


def test_independence_step_matches_oracle_chain_by_chain():
    """rtt_indep_mh on an FP64 handle with FP32 inference against the oracle's
    independence step (Sec. 3.3, Metropolis-Hastings on |psi|^2 with a
    proposal q): the same Philox proposals (divergent samples explained), and
    for every chain whose proposal agrees the same accept/reject decision,
    except where log u lies within the FP32 bound of the log acceptance ratio;
    accepted chains carry the FP64 amplitude of their new spins bit for bit."""
    rtt = _rtt()
    inst = inputs.make_instance(2, 5, 2, 8, 1.5, seed=61, mixing=True)
    N, H, B = inst.n_spins, 64, 2000
    o = orc.Oracle(inst)
    order = inst.path[:N].astype(np.int32)
    w = inputs.made_init_weights(62, N, H)
    p = made.masked_params(w, N, H)
    s_cur = inputs.initial_spins(63, B, N)
    chain0, rnd, seed = 5, 3, 64
    with rtt.RTT(inst, "fp64") as m, rtt.MADE(N, H, order, w, seed=seed) as mm:
        mm.set_inference(False)
        sg = torch.from_numpy(s_cur.copy()).cuda()
        _, _, st = m.log_amplitudes(sg)
        prop, lq_new = mm.sample(B, chain0=chain0, round=rnd)      # the proposals it draws
        lq_cur = mm.log_prob(sg)
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        rtt.indep_mh(m, mm, sg, st, rnd, acc, chain0=chain0)
        torch.cuda.synchronize()
        prop, lq_new, lq_cur = prop.cpu().numpy(), lq_new.cpu().numpy(), lq_cur.cpu().numpy()
        s_after, st_after, acc = sg.cpu().numpy(), st.cpu().numpy(), acc.cpu().numpy()
    so, lqo_new = made.sample(p, order, B, seed, chain0, rnd, N)
    same = check_sample_divergences(p, order, prop, so, seed, chain0, rnd)
    lqo_cur = made.log_prob(p, s_cur, order)
    la_cur, _, _, _ = o.log_amplitudes(s_cur)
    la_new, _, m_new, e_new = o.log_amplitudes(so)
    x_cur, _ = made.inputs_of(s_cur, order)
    x_new, _ = made.inputs_of(so, order)
    # log q carries at most the sum over positions of the logit bound
    tol = fp32_logit_bound(p, x_cur).sum(axis=1) + fp32_logit_bound(p, x_new).sum(axis=1) + 1e-9
    accepted_gpu = acc == 1
    assert np.array_equal(accepted_gpu, np.all(s_after == prop, axis=1) & np.any(prop != s_cur, axis=1)
                          | (accepted_gpu & np.all(prop == s_cur, axis=1)))
    n_checked = 0
    for c in np.flatnonzero(same):
        u = made.accept_uniform(seed, chain0 + c, rnd, N)
        dec_o = made.indep_mh_decide(la_cur[c], lqo_cur[c], la_new[c], lqo_new[c], u)
        if dec_o != accepted_gpu[c]:
            delta = 2.0 * (la_new[c] - la_cur[c]) + lqo_cur[c] - lqo_new[c]
            assert abs(np.log(u) - delta) <= tol[c], (c, np.log(u), delta, tol[c])
        n_checked += 1
        if accepted_gpu[c]:
            assert np.array_equal(s_after[c], so[c])
            assert st_after[c].view(np.float64)[0] == m_new[c] and st_after[c][1] == e_new[c]
        else:
            assert np.array_equal(s_after[c], s_cur[c])
    assert n_checked >= 0.9 * B and 0 < accepted_gpu.mean() < 1
