"""Pins of the replica-space oracle (Sec. 2.2.3 and Sec. 3.1).

Every check compares the oracle with something other than itself: the lifting
example printed in the paper, Pauli operators and the constraint C written as
index arithmetic on dense vectors, a dense TFIM matrix, closed-form
low-rank approximation errors, and the exact ground state.
"""
import os

import numpy as np
import pytest

from paper_2604_22718_gb300 import inputs
from oracle import replica as rp
from oracle import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hv_path():
    for line in open(os.path.join(GOLDEN, "psi_hv_example.txt")):
        f = line.split()
        if f and f[0] == "HV":
            return np.asarray([int(x) - 1 for x in f[1:]], dtype=np.int32)
    raise AssertionError("HV path missing from the fixture")


# ---- dense reference operations (index arithmetic, i_1 / spin 0 the most significant bit)

def _bits(n):
    idx = np.arange(1 << n, dtype=np.int64)
    return (idx[:, None] >> (n - 1 - np.arange(n))[None, :]) & 1


def _dense_pauli(v, n, sites_ops):
    """Apply prod_k P_k to a dense vector over n two-level sites."""
    idx = np.arange(1 << n, dtype=np.int64)
    out = v.copy()
    for k, op in sites_ops:
        b = n - 1 - int(k)
        if op == "X":
            out = out[idx ^ (1 << b)]
        elif op == "Z":
            out = out * (1 - 2 * ((idx >> b) & 1))
    return out


def _dense_C(phi_dense, path, n):
    """psi_s = phi_{i(s)}, i(s)_k = s_{path[k]} (Eq. rtt_equal_C_tt)."""
    s = _bits(n)
    L = len(path)
    i = s[:, np.asarray(path)]
    flat = (i * (1 << (L - 1 - np.arange(L)))[None, :]).sum(axis=1)
    return phi_dense[flat]


def _dense_tfim(n, bonds, J, h):
    I2, Z, X = np.eye(2), np.diag([1.0, -1.0]), np.array([[0.0, 1.0], [1.0, 0.0]])

    def op(site_ops):
        m = np.array([[1.0]])
        for i in range(n):
            m = np.kron(m, site_ops.get(i, I2))
        return m
    H = np.zeros((1 << n, 1 << n))
    for i, j in bonds:
        H += J * op({int(i): Z, int(j): Z})
    for i in range(n):
        H -= h * op({i: X})
    return H


def _ops_to_list(row):
    names = {1: "X", 2: "Z"}
    return [(k, names[int(o)]) for k, o in enumerate(row) if o]


def _tt_from_dense(x, L):
    """Exact TT of a dense vector by successive SVDs (no truncation)."""
    cores, r, rest = [], 1, x.reshape(1, -1)
    for k in range(L - 1):
        M = rest.reshape(r * 2, -1)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        keep = int(np.sum(S > 1e-14 * S[0]))
        cores.append(U[:, :keep].reshape(r, 2, keep))
        rest = S[:keep, None] * Vt[:keep]
        r = keep
    cores.append(rest.reshape(r, 2, 1))
    return cores


# ---- lifting

def test_lift_reproduces_the_printed_example():
    path = _hv_path()
    terms, want = [], []
    for line in open(os.path.join(GOLDEN, "lift_example_hv.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        lhs, rhs = line.split("=>")
        f = lhs.split()
        factors = [(int(t.split(":")[0]) - 1, t.split(":")[1]) for t in f[2:]]
        terms.append((float(f[0]), factors, int(f[1])))
        want.append(sorted((int(t.split(":")[0]) - 1, t.split(":")[1]) for t in rhs.split()))
    eta, ops = rp.lift(terms, path, 6)
    assert len(want) == 4 and np.all(eta == 1.0)
    for k in range(4):
        assert sorted(_ops_to_list(ops[k])) == want[k]


def test_lift_commutes_with_the_constraint_bruteforce():
    """C A-bar phi = A C phi for random X/Z strings and blocks, N = 6, L = 12."""
    path = _hv_path()
    rng = np.random.default_rng(5)
    phi = rng.standard_normal(1 << 12)
    for trial in range(12):
        nf = int(rng.integers(1, 4))
        spins = rng.choice(6, size=nf, replace=False)
        factors = [(int(j), str(rng.choice(["X", "Z"]))) for j in spins]
        block = int(rng.integers(0, 2))
        eta, ops = rp.lift([(1.7, factors, block)], path, 6)
        lhs = _dense_C(eta[0] * _dense_pauli(phi, 12, _ops_to_list(ops[0])), path, 6)
        rhs = 1.7 * _dense_pauli(_dense_C(phi, path, 6), 6, factors)
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind", ["H", "HV", "HVDDp"])
def test_lifted_tfim_commutes_with_the_constraint(kind):
    lx, ly = 2, 2
    order = ("V", "H", "D", "Dp")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    terms = inputs.hbar_terms(kind, lx, ly, 3.0, orderings=order, alpha=0.3)
    eta, ops = rp.lift(terms, path, 4)
    rng = np.random.default_rng(7)
    phi = rng.standard_normal(1 << 16)
    hphi = np.zeros_like(phi)
    for k in range(len(eta)):
        hphi += eta[k] * _dense_pauli(phi, 16, _ops_to_list(ops[k]))
    bonds = np.concatenate([inputs.direction_bonds(lx, ly, d) for d in ("H", "V")])
    H = _dense_tfim(4, bonds, 1.0, 3.0)
    if kind == "HVDDp":
        H += _dense_tfim(4, np.concatenate([inputs.direction_bonds(lx, ly, d) for d in ("D", "Dp")]),
                         0.3, 0.0)
    np.testing.assert_allclose(_dense_C(hphi, path, 4), H @ _dense_C(phi, path, 4), atol=1e-10)


def test_terms_sent_to_their_own_ordering_are_local():
    lx = ly = 6
    order = ("V", "H", "D", "Dp")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    for d in order:
        terms = inputs.replica_terms(lx, ly, order, [(d, 1.0, d)], 0.0)
        _, ops = rp.lift(terms, path, 36)
        sites = [np.nonzero(r)[0] for r in ops]
        gaps = [s[1] - s[0] for s in sites]
        # neighbours along an ordering's lines are next to each other on the path
        # except where the snake turns between lines
        assert sum(g == 1 for g in gaps) >= len(gaps) - (lx + ly), d
        assert all(np.all(s // 36 == order.index(d)) for s in sites)


def test_lift_rejects_bad_input():
    path = _hv_path()
    with pytest.raises(ValueError):
        rp.lift([(1.0, [(0, "Y")], 0)], path, 6)
    with pytest.raises(ValueError):
        rp.lift([(1.0, [(0, "Z"), (0, "Z")], 0)], path, 6)
    with pytest.raises(ValueError):
        rp.block_sites(np.asarray([0, 1, 2, 0, 0, 1]), 3)


# ---- TT algebra against dense vectors

def test_apply_string_and_sum_match_dense():
    rng = np.random.default_rng(11)
    L = 8
    a, b = rp.tt_random(rng, L, 3), rp.tt_random(rng, L, 2)
    ops = rng.integers(0, 3, size=L).astype(np.uint8)
    got = rp.tt_dense(rp.apply_string(a, ops, -0.7))
    want = -0.7 * _dense_pauli(rp.tt_dense(a), L, _ops_to_list(ops))
    np.testing.assert_allclose(got, want, atol=1e-13)
    np.testing.assert_allclose(rp.tt_dense(rp.tt_sum(a, b)), rp.tt_dense(a) + rp.tt_dense(b),
                               atol=1e-13)


def test_round_without_truncation_is_exact_and_right_orthonormal():
    rng = np.random.default_rng(12)
    L = 9
    a, b = rp.tt_random(rng, L, 3), rp.tt_random(rng, L, 3)
    s = rp.tt_sum(a, b)
    r = rp.tt_round(s, 6)
    x = rp.tt_dense(s)
    np.testing.assert_allclose(rp.tt_dense(r), x, atol=1e-12 * np.abs(x).max())
    for G in r[1:]:
        M = G.reshape(G.shape[0], -1)
        np.testing.assert_allclose(M @ M.T, np.eye(G.shape[0]), atol=1e-12)
    assert rp.tt_norm(r) == pytest.approx(np.linalg.norm(x), rel=1e-12)


def test_round_is_eckart_young_at_a_single_truncated_bond():
    """L = 4: bonds 1 and 3 have rank <= 2, so rank-2 rounding truncates only the
    middle unfolding, a 4x4 matrix with singular values 3, 2, 1, 0.5: the error
    must be sqrt(1 + 0.25) and the result of rank 2."""
    rng = np.random.default_rng(13)
    U, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    V, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    M = U @ np.diag([3.0, 2.0, 1.0, 0.5]) @ V.T
    x = M.reshape(-1)                       # i1 i2 | i3 i4, i1 most significant
    t = _tt_from_dense(x, 4)
    r = rp.tt_round(t, 2)
    y = rp.tt_dense(r)
    assert np.linalg.norm(x - y) == pytest.approx(np.sqrt(1.25), rel=1e-12)
    assert np.linalg.matrix_rank(y.reshape(4, 4), tol=1e-10) == 2


def test_round_error_bounds():
    rng = np.random.default_rng(14)
    L, chi = 10, 3
    t = rp.tt_random(rng, L, 8)
    x = rp.tt_dense(t)
    r, disc = rp.tt_round(t, chi, return_discarded=True)
    err = np.linalg.norm(x - rp.tt_dense(r))
    upper = np.sqrt(sum(float(np.sum(d ** 2)) for d in disc))
    assert err <= upper * (1 + 1e-10)
    lower = 0.0
    for k in range(1, L):
        S = np.linalg.svd(x.reshape(1 << k, -1), compute_uv=False)
        lower = max(lower, float(np.sqrt(np.sum(S[chi:] ** 2))))
    assert err >= lower * (1 - 1e-10)
    assert err <= np.sqrt(L - 1) * lower * (1 + 1e-10) + 1e-12   # TT-SVD quasi-optimality


# ---- the power step

def test_tree_levels():
    L = 6
    phi = rp.tt_ones(L)
    for K, want in [(1, 0), (2, 1), (5, 3), (8, 3), (96, 7)]:
        eta = np.ones(K)
        ops = np.zeros((K, L), dtype=np.uint8)
        _, _, lv = rp.power_step(phi, eta, ops, 0.1, 4, return_tree=True)
        assert lv == want


def test_one_step_without_truncation_is_one_minus_tau_h():
    lx, ly = 2, 2
    order = ("H", "V")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    eta, ops = rp.lift(inputs.hbar_terms("HV", lx, ly, 3.0, orderings=order), path, 4)
    rng = np.random.default_rng(15)
    phi = rp.tt_random(rng, 8, 16)
    new, nrm = rp.power_step(phi, eta, ops, 0.1, 16)
    H = _dense_tfim(4, inputs.open_bonds(lx, ly), 1.0, 3.0)
    psi = rp.constrained_amplitudes(phi, path, 4)
    want = (psi - 0.1 * H @ psi) / nrm
    np.testing.assert_allclose(rp.constrained_amplitudes(new, path, 4), want,
                               atol=1e-11 * np.abs(want).max())
    assert rp.tt_norm(new) == pytest.approx(1.0, rel=1e-12)


def test_untruncated_power_method_reaches_the_ground_state():
    lx, ly = 2, 2
    order = ("H", "V")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    eta, ops = rp.lift(inputs.hbar_terms("HV", lx, ly, 3.0, orderings=order), path, 4)
    phi, logn = rp.power(rp.tt_ones(8), eta, ops, 0.1, 16, 150)
    H = _dense_tfim(4, inputs.open_bonds(lx, ly), 1.0, 3.0)
    w, v = np.linalg.eigh(H)
    psi = rp.constrained_amplitudes(phi, path, 4)
    psi = psi / np.linalg.norm(psi)
    assert abs(psi @ v[:, 0]) == pytest.approx(1.0, abs=1e-9)
    assert psi @ H @ psi == pytest.approx(w[0], rel=1e-9)
    assert np.all(np.isfinite(logn))


def test_truncated_power_method_is_variational_and_ordered():
    """Rank-2 and rank-4 TTs on a 3x3 lattice (path V+H+D+D', L = 36), 20
    steps: every RTT energy lies above the exact ground state; sending the
    vertical bonds to the V ordering (H-bar_HV) does far better than keeping
    every bond on H (H-bar_H), the ordering the paper reports; a larger rank
    does better; and rounding every pairwise sum of the tree to the final rank
    (chi_tree = chi) instead of to 2 chi loses most of that accuracy."""
    lx = ly = 3
    order = ("V", "H", "D", "Dp")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    H = _dense_tfim(9, inputs.open_bonds(lx, ly), 1.0, 3.0)
    e0 = np.linalg.eigvalsh(H)[0]

    def energy(tt):
        psi = rp.constrained_amplitudes(tt, path, 9)
        return psi @ H @ psi / (psi @ psi)
    e_start = energy(rp.tt_ones(36))
    err = {}
    for kind, chi, ct in [("H", 2, None), ("HV", 2, None), ("HV", 4, None), ("HV", 2, 2)]:
        eta, ops = rp.lift(inputs.hbar_terms(kind, lx, ly, 3.0, orderings=order), path, 9)
        phi, _ = rp.power(rp.tt_ones(36), eta, ops, 0.1, chi, 20, chi_tree=ct)
        err[kind, chi, ct] = energy(phi) - e0
        assert err[kind, chi, ct] >= -1e-9
    assert err["HV", 2, None] < 0.05 * (e_start - e0)
    assert err["HV", 2, None] < 0.2 * err["H", 2, None]
    assert err["HV", 4, None] < 0.5 * err["HV", 2, None]
    assert err["HV", 2, 2] > 5 * err["HV", 2, None]


def test_tree_without_intermediate_truncation_is_one_rounding_of_the_exact_sum():
    """With chi_tree at least the rank of every pairwise sum, the tree loses
    nothing: the step equals rounding phi - tau sum_k eta_k P_k phi once."""
    lx, ly = 2, 2
    order = ("H", "V")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    eta, ops = rp.lift(inputs.hbar_terms("HV", lx, ly, 3.0, orderings=order), path, 4)
    rng = np.random.default_rng(17)
    phi = rp.tt_random(rng, 8, 2)
    got, _ = rp.power_step(phi, eta, ops, 0.1, 2, chi_tree=64)
    S = rp.apply_string(phi, ops[0], eta[0])
    for k in range(1, len(eta)):
        S = rp.tt_sum(S, rp.apply_string(phi, ops[k], eta[k]))
    want = rp.tt_round(rp.tt_sum(phi, rp.tt_scale(S, -0.1)), 2)
    want = rp.tt_scale(want, 1.0 / rp.tt_norm(want))
    np.testing.assert_allclose(rp.tt_dense(got), rp.tt_dense(want), atol=1e-10)


def test_padded_cores_feed_the_sampler_format():
    """padded(tt) with b_L = b_R = e_0 is the RTT the sampler takes: the C
    oracle's amplitudes equal C phi."""
    lx, ly = 2, 3
    order = ("H", "V")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    rng = np.random.default_rng(16)
    tt = rp.tt_random(rng, 12, 3)
    cores = rp.padded(tt, 3)
    e0 = np.zeros(3)
    e0[0] = 1.0
    inst = inputs.RTTInstance(n_spins=6, path=path.astype(np.int32), tensors=cores, b_left=e0,
                              b_right=e0.copy(), bonds=inputs.open_bonds(lx, ly), J=1.0, h=3.0)
    np.testing.assert_allclose(orc.Oracle(inst).all_amplitudes(),
                               rp.constrained_amplitudes(tt, path, 6), rtol=1e-12, atol=1e-14)
    back = rp.unpadded(cores)
    np.testing.assert_allclose(rp.tt_dense(back), rp.tt_dense(tt), atol=1e-14)
