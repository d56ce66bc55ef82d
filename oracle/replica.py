"""Replica- and physical-space optimization (Sec. 3.1, 3.2) in plain FP64 -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path (the CUDA library and
its Python binding) never calls it.

Objects (Sec. 2.2.3, "RTT as a tensor network"):
  * a TT phi over the replica space: L sites i_1..i_L in {0,1}, cores G_k of
    shape (r_{k-1}, 2, r_k) with r_0 = r_L = 1, phi_i = G_1[i_1] ... G_L[i_L];
  * the constraint C: psi_s = phi_{i(s)}, i(s)_k = s_{path[k]} (Eq. rtt_equal_C_tt);
  * a replica-space Pauli string: a coefficient eta and one of X, Z per site
    (identity elsewhere).

What it computes:
  * ``block_sites``: R_{j,c}, the train site of spin j in replica block c, for
    a path that is a concatenation of orderings (each a permutation of the spins).
  * ``lift``: A-bar from A (commutation rules of Sec. 2.2.3): Z_j goes to one
    replica of j (the block the term is sent to), X_j becomes X on every
    replica of j.  Y is not lifted (it would make the TT complex).
  * ``apply_string``: the rank-1 MPO eta * A-bar_k applied to a TT: X swaps the
    two physical slices of a core, Z negates its slice 1; eta scales core 1.
  * ``tt_sum``: the sum of two TTs (block-diagonal cores, first core
    concatenated along its right bond, last along its left bond).
  * ``tt_round``: compression to rank chi: left-to-right reduced QR of every
    core, then right-to-left truncated SVD keeping the chi largest singular
    values at every bond (fixed rank, no tolerance).
  * ``power_step``: one application of 1 - tau H-bar, in the order of Sec. 3.1:
    the terms eta_k A-bar_k phi, summed two by two with a compression after
    every sum (an odd last item passes to the next level unchanged) until one
    TT S is left; then phi' = compress(phi - tau S) to rank chi, scaled to unit
    replica-space 2-norm (RTTs are not normalised; the scale keeps the numbers
    finite).  The pairwise sums are compressed to chi_tree, by default 2 chi
    (the rank a sum of two rank-chi TTs has); chi_tree = chi truncates every
    pairwise sum to the final rank.

Physical-space optimization (Sec. 3.2, Sec. 4):
  * ``apply_operator``: phi^alpha = O-bar_alpha phi, the terms summed two by two
    with a rounding after every sum, the root rounded once more, scaled to unit
    norm (psi^alpha = O_alpha psi built "as in the replica-space optimization");
  * ``combine``: phi' = sum_alpha c_alpha phi^alpha (Eq. lin_comb) the same way.
  Pinned in ``tests/test_oracle_physical.py``: without truncation they are the
  dense operator and the dense linear combination; with H~, S~ enumerated
  exactly, the combination's energy is the lowest generalized eigenvalue, at
  most the starting energy (the identity is one of the operators) and at least
  the ground-state energy.

Parity status: pinned in ``tests/test_oracle_replica.py`` against the paper's
worked lifting example (``tests/golden/lift_example_hv.txt``), the identity
C A-bar phi = A C phi by brute force on dense vectors (N = 6), dense
Kronecker-product Pauli strings, dense sums, exact reconstruction when no
truncation is needed, the Eckart-Young best rank-chi approximation at a single
truncated bond, the TT-SVD error bound, and convergence of the untruncated
power method to the exact ground state of a dense TFIM matrix.
"""
from __future__ import annotations

import numpy as np

OPS = {"I": 0, "X": 1, "Z": 2}


# ---------------------------------------------------------------- lifting

def block_sites(path, n_spins):
    """R[j][c] = train site of spin j in block c (blocks of n_spins sites)."""
    path = np.asarray(path, dtype=np.int64)
    L = path.shape[0]
    if n_spins < 1 or L % n_spins:
        raise ValueError("path length is not a multiple of the number of spins")
    nb = L // n_spins
    R = np.full((n_spins, nb), -1, dtype=np.int64)
    for c in range(nb):
        blk = path[c * n_spins:(c + 1) * n_spins]
        if sorted(blk.tolist()) != list(range(n_spins)):
            raise ValueError(f"block {c} of the path is not a permutation of the spins")
        for pos, j in enumerate(blk):
            R[j, c] = c * n_spins + pos
    return R


def lift(terms, path, n_spins):
    """Replica-space strings of sum_k coef_k prod_f P_f(spin_f).

    terms: iterable of (coef, factors, block) with factors a list of
    (spin, 'X' | 'Z'), all spins of a term distinct; block = the replica that
    the term's Z factors are sent to.  Returns (eta [K], ops [K][L] uint8)."""
    R = block_sites(path, n_spins)
    L = len(path)
    etas, rows = [], []
    for coef, factors, block in terms:
        row = np.zeros(L, dtype=np.uint8)
        spins = [int(j) for j, _ in factors]
        if len(set(spins)) != len(spins):
            raise ValueError("a term names one spin twice")
        for j, op in factors:
            if op == "Z":
                row[R[j, block]] = OPS["Z"]
            elif op == "X":
                row[R[j, :]] = OPS["X"]
            else:
                raise ValueError(f"Pauli {op!r} is not lifted (real TTs only)")
        etas.append(float(coef))
        rows.append(row)
    return np.asarray(etas, dtype=np.float64), np.asarray(rows, dtype=np.uint8).reshape(-1, L)


# ---------------------------------------------------------------- TT algebra

def tt_ones(L):
    """phi_i = 1 for every i: rank-1 cores of ones (the paper's phi^(0))."""
    return [np.ones((1, 2, 1)) for _ in range(L)]


def tt_random(rng, L, chi):
    """Gaussian cores with ranks min(chi, 2^k, 2^(L-k))."""
    r = [min(chi, 2 ** k, 2 ** (L - k)) for k in range(L + 1)]
    return [rng.standard_normal((r[k], 2, r[k + 1])) for k in range(L)]


def apply_string(tt, ops, eta):
    out = []
    for k, G in enumerate(tt):
        G = G.copy()
        if ops[k] == OPS["X"]:
            G = G[:, ::-1, :].copy()
        elif ops[k] == OPS["Z"]:
            G[:, 1, :] = -G[:, 1, :]
        out.append(G)
    out[0] = eta * out[0]
    return out


def tt_sum(a, b):
    L = len(a)
    if L == 1:
        return [a[0] + b[0]]
    out = []
    for k in range(L):
        A, B = a[k], b[k]
        if k == 0:
            G = np.concatenate([A, B], axis=2)
        elif k == L - 1:
            G = np.concatenate([A, B], axis=0)
        else:
            G = np.zeros((A.shape[0] + B.shape[0], 2, A.shape[2] + B.shape[2]))
            G[:A.shape[0], :, :A.shape[2]] = A
            G[A.shape[0]:, :, A.shape[2]:] = B
        out.append(G)
    return out


def tt_scale(tt, c):
    out = [G.copy() for G in tt]
    out[0] = c * out[0]
    return out


def tt_round(tt, chi, return_discarded=False):
    """Left-to-right QR, then right-to-left SVD truncated to chi."""
    L = len(tt)
    cores = [G.copy() for G in tt]
    for k in range(L - 1):
        r0, _, r1 = cores[k].shape
        Q, Rm = np.linalg.qr(cores[k].reshape(r0 * 2, r1), mode="reduced")
        cores[k] = Q.reshape(r0, 2, Q.shape[1])
        cores[k + 1] = np.einsum("ab,bsc->asc", Rm, cores[k + 1])
    discarded = []
    for k in range(L - 1, 0, -1):
        r0, _, r1 = cores[k].shape
        U, S, Vt = np.linalg.svd(cores[k].reshape(r0, 2 * r1), full_matrices=False)
        t = min(chi, S.shape[0])
        discarded.append(S[t:].copy())
        cores[k] = Vt[:t].reshape(t, 2, r1)
        cores[k - 1] = np.einsum("asb,bc->asc", cores[k - 1], U[:, :t] * S[:t])
    if return_discarded:
        return cores, discarded[::-1]
    return cores


def tt_norm(tt):
    E = np.ones((1, 1))
    for G in tt:
        E = np.einsum("ab,asc,bsd->cd", E, G, G)
    return float(np.sqrt(E[0, 0]))


def tt_eval(tt, idx):
    """phi at replica configurations idx [B][L] (0/1)."""
    idx = np.asarray(idx)
    out = np.empty(idx.shape[0])
    for b in range(idx.shape[0]):
        v = np.ones(1)
        for k, G in enumerate(tt):
            v = v @ G[:, int(idx[b, k]), :]
        out[b] = v[0]
    return out


def tt_dense(tt):
    """phi as a dense vector over 2^L, i_1 the most significant bit."""
    v = np.ones((1, 1))
    for G in tt:
        v = np.einsum("ia,asb->isb", v, G).reshape(-1, G.shape[2])
    return v[:, 0]


def constrained_amplitudes(tt, path, n_spins):
    """psi = C phi on all 2^N physical configurations (spin 0 the MSB)."""
    idx = np.arange(1 << n_spins, dtype=np.int64)
    spins = (idx[:, None] >> (n_spins - 1 - np.arange(n_spins))[None, :]) & 1
    return tt_eval(tt, spins[:, np.asarray(path)])


def tree_rank(chi, chi_tree=None):
    """Rank the tree's pairwise sums are rounded to: 2 chi (the rank of a sum of
    two rank-chi TTs) unless given."""
    return 2 * chi if chi_tree is None else int(chi_tree)


def power_step(phi, eta, ops, tau, chi, return_tree=False, chi_tree=None):
    """phi' = compress(phi - tau * S) / norm, S = tree sum of eta_k A-bar_k phi
    with every pairwise sum rounded to chi_tree (default 2 chi) and phi' to chi."""
    ct = tree_rank(chi, chi_tree)
    items = [apply_string(phi, ops[k], eta[k]) for k in range(len(eta))]
    levels = 0
    while len(items) > 1:
        nxt = [tt_round(tt_sum(items[i], items[i + 1]), ct) for i in range(0, len(items) - 1, 2)]
        if len(items) % 2:
            nxt.append(items[-1])
        items = nxt
        levels += 1
    out = tt_round(tt_sum(phi, tt_scale(items[0], -tau)), chi)
    nrm = tt_norm(out)
    out = tt_scale(out, 1.0 / nrm)
    if return_tree:
        return out, nrm, levels
    return out, nrm


def power(phi, eta, ops, tau, chi, steps, chi_tree=None):
    log_norms = []
    for _ in range(steps):
        phi, nrm = power_step(phi, eta, ops, tau, chi, chi_tree=chi_tree)
        log_norms.append(np.log(nrm))
    return phi, np.asarray(log_norms)


def padded(tt, chi):
    """Cores zero-padded to [L][2][chi][chi] (row = left bond), the layout the
    RTT sampler takes with b_L = b_R = e_0."""
    L = len(tt)
    out = np.zeros((L, 2, chi, chi))
    for k, G in enumerate(tt):
        r0, _, r1 = G.shape
        out[k, :, :r0, :r1] = np.transpose(G, (1, 0, 2))
    return out


def unpadded(cores):
    """Inverse of padded: cores [L][2][chi][chi] -> list of (chi, 2, chi)
    (first core's left rank and last core's right rank cut to 1)."""
    L = cores.shape[0]
    out = []
    for k in range(L):
        G = np.transpose(cores[k], (1, 0, 2))
        if k == 0:
            G = G[:1]
        if k == L - 1:
            G = G[:, :, :1]
        out.append(np.ascontiguousarray(G))
    return out


# ---------------------------------------------------------------- physical-space optimization

def tree_round(items, chi, chi_tree=None):
    """Sum of TTs, two by two with a rounding to chi_tree (default 2 chi) after
    every sum (an odd last item passes up unchanged), as in the replica-space
    step; the root is rounded to chi."""
    ct = tree_rank(chi, chi_tree)
    items = list(items)
    while len(items) > 1:
        nxt = [tt_round(tt_sum(items[i], items[i + 1]), ct) for i in range(0, len(items) - 1, 2)]
        if len(items) % 2:
            nxt.append(items[-1])
        items = nxt
    return tt_round(items[0], chi)


def normalised(tt):
    nrm = tt_norm(tt)
    return tt_scale(tt, 1.0 / nrm), nrm


def apply_operator(phi, eta, ops, chi, chi_tree=None):
    """phi^alpha = O-bar_alpha phi (Sec. 3.2: psi^alpha = O_alpha psi built with
    O-bar_alpha as in the replica-space optimization), rounded to chi and scaled
    to unit replica-space norm.  Returns (phi^alpha, norm before scaling).  The
    physical-space step keeps the states at twice the rank of phi (Sec. 3.2
    compresses only the final combination) and calls this with chi = 2 chi_phi,
    chi_tree = 4 chi_phi."""
    return normalised(tree_round([apply_string(phi, ops[k], eta[k]) for k in range(len(eta))], chi,
                                 chi_tree))


def combine(phis, coef, chi, chi_tree=None):
    """phi' = sum_alpha c_alpha phi^alpha (Eq. lin_comb, the TTs summed back into
    one), rounded to chi and scaled to unit norm."""
    return normalised(tree_round([tt_scale(p, float(c)) for p, c in zip(phis, coef)], chi, chi_tree))
