"""Pins of the FP64 oracle of the learned proposal (CPU only): normalisation
by enumeration, the autoregressive property, gradients against central finite
differences, Adam against torch.optim.Adam, sampling against the enumerated
distribution, and the independence Metropolis-Hastings rule against an exact
proposal (acceptance identically one)."""
import itertools

import numpy as np
import pytest

from oracle import made
from oracle import oracle as orc
from paper_2604_22718_gb300 import inputs


def _all(n):
    return np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)


def _params(N, H, seed=1):
    p = made.masked_params(inputs.made_init_weights(seed, N, H), N, H)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.3   # nonzero biases exercise them
    return p


def test_probabilities_sum_to_one():
    N, H = 8, 16
    p = _params(N, H)
    order = np.random.default_rng(0).permutation(N)
    lq = made.log_prob(p, _all(N), order)
    assert np.sum(np.exp(lq)) == pytest.approx(1.0, abs=1e-12)


def test_autoregressive_property_exact():
    N, H = 7, 12
    p = _params(N, H, seed=2)
    rng = np.random.default_rng(3)
    x = rng.choice([-1.0, 1.0], size=(5, N))
    base = made.forward(p, x)[4]
    for dprime in range(N):
        y = x.copy()
        y[:, dprime] = -y[:, dprime]
        out = made.forward(p, y)[4]
        # logits at positions d <= dprime never see input dprime
        assert np.array_equal(out[:, :dprime + 1], base[:, :dprime + 1])
    # and logit 0 is the bias alone
    assert np.array_equal(base[:, 0], np.full(5, p["b3"][0]))


def test_gradients_match_central_differences():
    N, H, B = 6, 10, 5
    p = _params(N, H, seed=4)
    order = np.arange(N)[::-1].copy()
    spins = np.random.default_rng(5).integers(0, 2, (B, N)).astype(np.uint8)
    _, g = made.nll_and_grads(p, spins, order, N, H)
    M = dict(zip(("W1", "W2", "W3"), made.masks(N, H)))
    rng = np.random.default_rng(6)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[name].shape)
            if name in M and M[name][idx] == 0:
                assert g[name][idx] == 0.0
                continue
            pp, pm = dict(p), dict(p)
            pp[name] = p[name].copy()
            pm[name] = p[name].copy()
            pp[name][idx] += h
            pm[name][idx] -= h
            fd = (made.nll_and_grads(pp, spins, order, N, H)[0] -
                  made.nll_and_grads(pm, spins, order, N, H)[0]) / (2 * h)
            assert g[name][idx] == pytest.approx(fd, rel=1e-6, abs=1e-9), (name, idx)
    for name in M:
        assert np.all(g[name][M[name] == 0] == 0.0)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    N, H, B = 5, 8, 7
    p = _params(N, H, seed=7)
    order = np.arange(N)
    rng = np.random.default_rng(8)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    opt = torch.optim.Adam(list(tp.values()), lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(vv) for k, vv in p.items()}
    for step in range(1, 4):
        spins = rng.integers(0, 2, (B, N)).astype(np.uint8)
        _, g = made.nll_and_grads(p, spins, order, N, H)
        p, m, v = made.adam_step(p, g, m, v, step)
        opt.zero_grad()
        for k in tp:
            tp[k].grad = torch.tensor(g[k], dtype=torch.float64)
        opt.step()
    for k in p:
        np.testing.assert_allclose(p[k], tp[k].detach().numpy(), rtol=1e-12, atol=1e-15)


def test_sampling_follows_q_and_reports_its_log_prob():
    scipy_stats = pytest.importorskip("scipy.stats")
    N, H, B = 6, 12, 12000
    p = _params(N, H, seed=9)
    order = np.array([2, 0, 5, 1, 4, 3])
    spins, lq = made.sample(p, order, B, seed=11, chain0=0, rnd=3, N=N)
    np.testing.assert_allclose(lq, made.log_prob(p, spins, order), rtol=1e-12, atol=1e-12)
    allc = _all(N)
    q = np.exp(made.log_prob(p, allc, order))
    idx = (spins.astype(np.int64) * (1 << np.arange(N - 1, -1, -1))).sum(axis=1)
    obs = np.bincount(idx, minlength=1 << N)
    keep = q * B >= 5
    o_b, e_b = obs[keep].astype(float), q[keep] * B
    if np.any(~keep):
        o_b, e_b = np.append(o_b, obs[~keep].sum()), np.append(e_b, q[~keep].sum() * B)
    e_b *= o_b.sum() / e_b.sum()
    chi2, pval = scipy_stats.chisquare(o_b, e_b)
    assert pval > 1e-3


def test_independence_mh_with_exact_proposal_always_accepts():
    inst = inputs.make_instance(2, 3, 2, 3, 3.0, seed=12, mixing=False)
    o = orc.Oracle(inst)
    allc = _all(6)
    la, _, _, _ = o.log_amplitudes(allc)
    logZ = np.log(np.sum(np.exp(2 * la)))
    logP = 2 * la - logZ
    rng = np.random.default_rng(13)
    for _ in range(200):
        a, b = rng.integers(0, 64, 2)
        u = orc.uniform_keyed(5, made.MADE_STREAM, int(a), int(b), 6)
        assert made.indep_mh_decide(la[a], logP[a], la[b], logP[b], u)
