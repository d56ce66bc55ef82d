"""Checks shared by the GPU parity tests (a helper module, not collected).

Floating-point bounds (Sec. 2.2.1 Eq. RTT evaluated site by site):
every site product v A_k of a row carries a componentwise error of at most
eps (|v||A_k|)_b, so log|psi| moves by at most eps (sum_k kappa_k + kappa_fin)
= eps K(s) to first order, with the conditioning numbers of the FP64 oracle
(orc_amplitude_cond).  A ratio psi(s')/psi(s) therefore carries at most
|r| eps (K(s) + K(s')), its square twice that.

  split precision (BF16 or FP16 hi/lo, three products, FP32 accumulation):
      eps = 3 u_b^2 + chi u_32
  FP32 CUDA cores (chi fma terms):  eps = (chi + 1) u_32
"""
import numpy as np

U32 = 2.0 ** -24
UB = {"bf16x3": 2.0 ** -8, "fp16x3": 2.0 ** -11}


def eps_site(chi: int, prec: str) -> float:
    if prec in UB:
        return 3 * UB[prec] ** 2 + chi * U32
    if prec == "fp32":
        return (chi + 1) * U32
    return (chi + 1) * 2.0 ** -53


def amplitude_K(o, spins) -> np.ndarray:
    """K(s) = sum_k kappa_k + kappa_fin per configuration (FP64 oracle)."""
    c = o.amplitude_cond(np.ascontiguousarray(spins, dtype=np.uint8))
    return c[:, 0] + c[:, 2]


def check_sweep_divergences(o, seed, s0, s1, sweep, eps, chain0=0, slack=0.0, threads=16):
    """One sweep of the GPU took every chain from s0 to s1.  The oracle
    replays it, following the recorded decisions (Sec. 3.3: proposal j flips
    spin path[j]; a sweep proposes every spin once).  Every proposal at which
    the recorded decision differs from the FP64 rule u < r^2 at the same state
    must be a near tie: |u - r^2| <= 2 r^2 eps (K(s) + K(s')) + slack, the
    slack covering a decision the kernel takes on a shortened uniform.  No
    divergence is left unexplained.  Returns (proposals, divergences, largest
    |u - r^2| / tolerance among them)."""
    r2, u, taken, rule, states = o.replay_sweep(seed, s0, s1, sweep, chain0=chain0,
                                                threads=threads)
    div = np.argwhere(taken != rule)
    worst = 0.0
    if len(div):
        s = np.stack([states[c, j] for c, j in div])
        sf = s.copy()
        for k, (c, j) in enumerate(div):
            sf[k, int(o.path[j])] ^= 1
        K = amplitude_K(o, s) + amplitude_K(o, sf)
        rr = r2[div[:, 0], div[:, 1]]
        gap = np.abs(u[div[:, 0], div[:, 1]] - rr)
        tol = 2.0 * rr * eps * K + slack
        worst = float(np.max(gap / tol))
        assert np.all(gap <= tol), (
            f"unexplained divergences at (chain, proposal) {div[gap > tol].tolist()[:8]}: "
            f"|u - r^2| {gap[gap > tol][:8]}, tolerance {tol[gap > tol][:8]}")
    return int(taken.size), int(len(div)), worst


def local_energy_bound(o, spins, ratios, eps, J, h, n_bonds):
    """Per configuration, a bound on |E_loc(split) - E_loc(FP64)|: the ZZ term
    is exact; every ratio carries |r_i| eps (K(s) + K(s^(i))); plus the FP64
    rounding of the sums."""
    spins = np.ascontiguousarray(spins, dtype=np.uint8)
    B, N = spins.shape
    K = amplitude_K(o, spins)
    flipped = np.repeat(spins, N, axis=0)
    flipped[np.arange(B * N), np.tile(np.arange(N), B)] ^= 1
    Kf = amplitude_K(o, flipped).reshape(B, N)
    dr = np.abs(ratios) * eps * (K[:, None] + Kf)
    return abs(h) * dr.sum(axis=1) + 1e-12 * (abs(J) * n_bonds + abs(h) * np.abs(ratios).sum(axis=1))
