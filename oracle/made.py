"""FP64 oracle of the learned independence proposal -- TEST INFRASTRUCTURE ONLY.

A MADE (masked autoencoder for distribution estimation, Germain, Gregor,
Murray and Larochelle, ICML 2015): an autoregressive masked MLP with two ReLU
hidden layers whose output d is the conditional q(t_d = 1 | t_<d) = sigmoid
(logit_d) of the bit t_d = s_order[d].  It proposes configurations s' ~ q for
an independence Metropolis-Hastings step on P = |psi|^2 / Z (Sec. 3.3):
accept with min(1, |psi(s')|^2 q(s) / (|psi(s)|^2 q(s'))).

Conventions (shared with the CUDA kernels by definition, not by code):
  order[d]     spin at autoregressive position d (the order of the first N
               train sites);  input x_d = 1 - 2 s_order[d]  (+-1)
  degrees      input d -> d+1 (1..N); hidden unit k -> (k mod (N-1)) + 1
               (round-robin, N > 1; all 1 if N = 1); output d -> d+1
  masks        W1[k,d] kept iff m1_k >= d+1;  W2[k2,k1] iff m2_k2 >= m1_k1;
               W3[d,k] iff d+1 > m2_k   (so logit_0 is the bias alone)
  parameters   packed flat in the order W1 [H,N], b1 [H], W2 [H,H], b2 [H],
               W3 [N,H], b3 [N] (row-major)
  loss         NLL = -mean_b log q(s_b),  log q = sum_d log sigmoid((2t_d-1) logit_d)
  Adam         lr, beta1, beta2, eps on the masked gradient
  sampling     position d: u = Philox4x64-10(key (seed, 0x4D414445), counter
               (chain, round, d, 0)) -> t_d = [u < sigmoid(logit_d)];
               acceptance uniform at position N of the same counter family
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as orc

MADE_STREAM = 0x4D414445


def degrees(N: int, H: int):
    din = np.arange(1, N + 1)
    m = (np.arange(H) % (N - 1)) + 1 if N > 1 else np.ones(H, dtype=np.int64)
    return din, m, m.copy()


def masks(N: int, H: int):
    din, m1, m2 = degrees(N, H)
    M1 = (m1[:, None] >= din[None, :]).astype(np.float64)
    M2 = (m2[:, None] >= m1[None, :]).astype(np.float64)
    M3 = (din[:, None] > m2[None, :]).astype(np.float64)
    return M1, M2, M3


def shapes(N, H):
    return [("W1", (H, N)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (N, H)), ("b3", (N,))]


def unpack(flat, N, H):
    out, o = {}, 0
    for name, shp in shapes(N, H):
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(p, N, H):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in shapes(N, H)])


def apply_masks(p, N, H):
    M1, M2, M3 = masks(N, H)
    q = dict(p)
    q["W1"] = p["W1"] * M1
    q["W2"] = p["W2"] * M2
    q["W3"] = p["W3"] * M3
    return q


def inputs_of(spins, order):
    s = np.asarray(spins, dtype=np.float64)[:, order]
    return 1.0 - 2.0 * s, s


def forward(p, x):
    a1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    logits = h2 @ p["W3"].T + p["b3"]
    return a1, h1, a2, h2, logits


def log_sigmoid(y):
    return np.minimum(y, 0.0) - np.log1p(np.exp(-np.abs(y)))


def log_prob(p, spins, order):
    x, t = inputs_of(spins, order)
    logits = forward(p, x)[4]
    return np.sum(log_sigmoid((2.0 * t - 1.0) * logits), axis=1)


def nll_and_grads(p, spins, order, N, H):
    """Mean NLL over the batch and its gradient (masked), by the chain rule."""
    x, t = inputs_of(spins, order)
    B = x.shape[0]
    a1, h1, a2, h2, logits = forward(p, x)
    nll = -np.mean(np.sum(log_sigmoid((2.0 * t - 1.0) * logits), axis=1))
    sig = 1.0 / (1.0 + np.exp(-logits))
    d3 = (sig - t) / B                      # dNLL/dlogits
    M1, M2, M3 = masks(N, H)
    g = {}
    g["W3"] = (d3.T @ h2) * M3
    g["b3"] = d3.sum(axis=0)
    dh2 = (d3 @ p["W3"]) * (a2 > 0)
    g["W2"] = (dh2.T @ h1) * M2
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2"]) * (a1 > 0)
    g["W1"] = (dh1.T @ x) * M1
    g["b1"] = dh1.sum(axis=0)
    return nll, g


def adam_step(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction; step >= 1."""
    out_p, out_m, out_v = {}, {}, {}
    for k in p:
        out_m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        out_v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k]
        mh = out_m[k] / (1 - beta1 ** step)
        vh = out_v[k] / (1 - beta2 ** step)
        out_p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return out_p, out_m, out_v


def sample(p, order, B, seed, chain0, rnd, N):
    """Ancestral sampling position by position; returns (spins [B][N], log q)."""
    spins = np.zeros((B, N), dtype=np.uint8)
    x = np.zeros((B, N))
    logq = np.zeros(B)
    for d in range(N):
        logit = forward(p, x)[4][:, d]
        pr = 1.0 / (1.0 + np.exp(-logit))
        u = np.array([orc.uniform_keyed(seed, MADE_STREAM, chain0 + c, rnd, d) for c in range(B)])
        t = (u < pr).astype(np.float64)
        logq += log_sigmoid((2.0 * t - 1.0) * logit)
        spins[:, order[d]] = t.astype(np.uint8)
        x[:, d] = 1.0 - 2.0 * t
    return spins, logq


def accept_uniform(seed, chain, rnd, N):
    return orc.uniform_keyed(seed, MADE_STREAM, chain, rnd, N)


def indep_mh_decide(log_abs_cur, logq_cur, log_abs_new, logq_new, u):
    """accept iff log u < 2 (log|psi'| - log|psi|) + log q(s) - log q(s')."""
    return math.log(u) < 2.0 * (log_abs_new - log_abs_cur) + logq_cur - logq_new if u > 0 else True


def masked_params(flat_unmasked, N, H):
    """Unpack an (unmasked) flat parameter vector and apply the masks."""
    return apply_masks(unpack(flat_unmasked, N, H), N, H)
