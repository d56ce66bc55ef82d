"""Pins of the physical-space optimization oracle (Sec. 3.2, Sec. 4).

The operators psi^alpha = O_alpha psi, the optimal combination of Eq. lin_comb
through the generalized eigenproblem Eq. gen_eig1, and the TT that carries it,
checked against dense matrices on lattices small enough to enumerate.
"""
import numpy as np
import pytest

from paper_2604_22718_gb300 import inputs
from oracle import dual
from oracle import replica as rp


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


def _setup(lx=3, ly=2, order=("H", "V")):
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    N = lx * ly
    ops_list = [
        ("1", [(1.0, [], 0)]),
        ("X", inputs.replica_terms(lx, ly, order, [], 1.0)),                 # -O_X
        ("ZZ_HV", inputs.replica_terms(lx, ly, order, [("H", 1.0, "H"), ("V", 1.0, "V")], 0.0)),
    ]
    lifted = [rp.lift(t, path, N) for _, t in ops_list]
    return path, N, lifted


def _dense_op(n, terms):
    """A physical operator sum_k coef_k prod P from its term list."""
    I2, Z, X = np.eye(2), np.diag([1.0, -1.0]), np.array([[0.0, 1.0], [1.0, 0.0]])
    A = np.zeros((1 << n, 1 << n))
    for coef, factors, _ in terms:
        d = {int(j): (Z if op == "Z" else X) for j, op in factors}
        m = np.array([[1.0]])
        for i in range(n):
            m = np.kron(m, d.get(i, I2))
        A += coef * m
    return A


def test_apply_operator_without_truncation_is_the_operator():
    lx, ly, order = 3, 2, ("H", "V")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    terms = inputs.replica_terms(lx, ly, order, [("H", 0.7, "H"), ("V", -1.1, "V")], 2.0)
    eta, ops = rp.lift(terms, path, 6)
    rng = np.random.default_rng(2)
    phi = rp.tt_random(rng, 12, 3)
    out, nrm = rp.apply_operator(phi, eta, ops, 64)
    want = _dense_op(6, terms) @ rp.constrained_amplitudes(phi, path, 6)
    got = rp.constrained_amplitudes(out, path, 6) * nrm
    np.testing.assert_allclose(got, want, atol=1e-11 * np.abs(want).max())
    assert rp.tt_norm(out) == pytest.approx(1.0, rel=1e-12)


def test_identity_operator_keeps_the_state():
    path, N, lifted = _setup()
    rng = np.random.default_rng(3)
    phi = rp.tt_random(rng, 12, 2)
    out, nrm = rp.apply_operator(phi, *lifted[0], 2)
    np.testing.assert_allclose(rp.tt_dense(out) * nrm, rp.tt_dense(phi), atol=1e-12)


def test_combine_without_truncation_is_the_linear_combination():
    rng = np.random.default_rng(4)
    phis = [rp.tt_random(rng, 10, 2) for _ in range(3)]
    c = np.array([0.3, -1.2, 2.0])
    out, nrm = rp.combine(phis, c, 8)
    want = sum(ci * rp.tt_dense(p) for ci, p in zip(c, phis))
    np.testing.assert_allclose(rp.tt_dense(out) * nrm, want, atol=1e-12 * np.abs(want).max())


def test_optimal_combination_energy_is_lambda_and_never_above_the_start():
    """Exact H~, S~ by enumeration over the states psi^alpha: the lowest
    eigenvalue equals the energy of sum c_alpha psi^alpha (uncompressed), and it
    is at most the energy of psi^1 = psi (the identity is among the operators)."""
    lx, ly, order = 3, 2, ("H", "V")
    path, N, lifted = _setup(lx, ly, order)
    rng = np.random.default_rng(5)
    phi = rp.tt_random(rng, 12, 2)
    phis = [rp.apply_operator(phi, e, o, 2)[0] for e, o in lifted]
    H = _dense_tfim(N, inputs.open_bonds(lx, ly), 1.0, 3.0)
    states = []
    e_l = np.zeros(2)
    e_l[0] = 1.0
    for p in phis:
        states.append(inputs.RTTInstance(n_spins=N, path=path.astype(np.int32),
                                         tensors=rp.padded(p, 2), b_left=e_l, b_right=e_l.copy(),
                                         bonds=inputs.open_bonds(lx, ly), J=1.0, h=3.0))
    Ht, St = dual.exact_tilde_matrices(states)
    w, c = dual.solve(Ht, St)
    lam = w.real[0]
    out, _ = rp.combine(phis, c, 64)               # no truncation
    psi = rp.constrained_amplitudes(out, path, N)
    assert psi @ H @ psi / (psi @ psi) == pytest.approx(lam, rel=1e-9)
    psi1 = rp.constrained_amplitudes(phis[0], path, N)
    assert lam <= psi1 @ H @ psi1 / (psi1 @ psi1) + 1e-10
    assert lam >= np.linalg.eigvalsh(H)[0] - 1e-9


def test_states_at_twice_the_rank_give_table1_pattern():
    """The reading of Sec. 3.2 the physical step takes (operator states kept at
    rank 2 chi, only the combination compressed to chi), on 3x3 with the
    Sec. 4 path and operators, exact H~ and S~: the step gains an order of
    magnitude over the start, and only with O_ZZ,DD' among the operators; the
    compression then costs little, as Table 1 and Sec. 4.3 find.  With the
    states themselves compressed to chi the gain is lost."""
    lx = ly = 3
    N = lx * ly
    order = ("V", "H", "D", "Dp")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    H = _dense_tfim(N, inputs.open_bonds(lx, ly), 1.0, 3.0)
    e0 = np.linalg.eigvalsh(H)[0]

    def err(tt):
        p = rp.constrained_amplitudes(tt, path, N)
        return (p @ H @ p / (p @ p) - e0) / abs(e0)

    eta, ops = rp.lift(inputs.hbar_terms("HV", lx, ly, 3.0, orderings=order), path, N)
    phi, _ = rp.power(rp.tt_ones(len(path)), eta, ops, 0.1, 2, 20)
    start = err(phi)
    operators = [
        [],
        inputs.replica_terms(lx, ly, order, [], 1.0),
        inputs.replica_terms(lx, ly, order, [("H", 1.0, "H"), ("V", 1.0, "V")], 0.0),
        inputs.replica_terms(lx, ly, order, [("D", 1.0, "D"), ("Dp", 1.0, "Dp")], 0.0),
    ]

    def step(ops_list, rank):
        phis = [rp.normalised(phi)[0] if not t else rp.apply_operator(phi, *rp.lift(t, path, N), rank)[0]
                for t in ops_list]
        P = np.stack([rp.constrained_amplitudes(p, path, N) for p in phis], axis=1)
        Z = np.sum(P * P, axis=0)
        w, c = dual.solve((P.T @ H @ P) / Z[:, None], (P.T @ P) / Z[:, None])
        return (w.real[0] - e0) / abs(e0), err(rp.combine(phis, c, 2)[0])

    lam4, new4 = step(operators, 4)
    assert new4 < 0.15 * start and new4 < 1.5 * lam4
    _, new2 = step(operators, 2)
    assert new2 > 0.5 * start
    _, nodd4 = step(operators[:3], 4)
    assert nodd4 > 0.5 * start


def test_exact_gram_schmidt_states_beat_compressed_ones():
    """The reading of Sec. 3.3 the physical step takes: the Gram-Schmidt
    states psi'^m = psi^m - S~_1m psi^1 enter the eigenproblem exactly (as
    direct sums) rather than compressed to chi.  On 3x3 with exact H~, S~ one
    iteration then gains an order of magnitude; compressing the new states to
    chi first keeps well under half of that gain."""
    lx = ly = 3
    N = lx * ly
    order = ("V", "H", "D", "Dp")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    H = _dense_tfim(N, inputs.open_bonds(lx, ly), 1.0, 3.0)
    e0 = np.linalg.eigvalsh(H)[0]

    def amp(tt):
        return rp.constrained_amplitudes(tt, path, N)

    def err(p):
        return (p @ H @ p / (p @ p) - e0) / abs(e0)

    eta, ops = rp.lift(inputs.hbar_terms("HV", lx, ly, 3.0, orderings=order), path, N)
    phi, _ = rp.power(rp.tt_ones(len(path)), eta, ops, 0.1, 2, 20)
    terms = [[], inputs.replica_terms(lx, ly, order, [], 1.0),
             inputs.replica_terms(lx, ly, order, [("H", 1.0, "H"), ("V", 1.0, "V")], 0.0),
             inputs.replica_terms(lx, ly, order, [("D", 1.0, "D"), ("Dp", 1.0, "Dp")], 0.0)]
    phis = [rp.normalised(rp.tt_round(phi, 4))[0] if not t
            else rp.apply_operator(phi, *rp.lift(t, path, N), 4, chi_tree=8)[0] for t in terms]
    P = np.stack([amp(p) for p in phis], axis=1)
    Z = np.sum(P * P, axis=0)
    St = (P.T @ P) / Z[:, None]
    T = dual.gram_schmidt(St, first_only=True)
    Q = P @ T.T                                      # the exact direct sums psi' = T psi
    Zq = np.sum(Q * Q, axis=0)
    _, cq = dual.solve((Q.T @ H @ Q) / Zq[:, None], (Q.T @ Q) / Zq[:, None])
    exact = err(amp(rp.combine(phis, T.T @ cq, 2)[0]))
    gs = [rp.normalised(rp.tt_round(phis[0], 2))[0]] + [
        rp.normalised(rp.tt_round(rp.tt_sum(phis[m], rp.tt_scale(phis[0], -St[0, m])), 2))[0]
        for m in range(1, 4)]
    G = np.stack([amp(p) for p in gs], axis=1)
    Zg = np.sum(G * G, axis=0)
    _, cg = dual.solve((G.T @ H @ G) / Zg[:, None], (G.T @ G) / Zg[:, None])
    compressed = err(amp(rp.combine(gs, cg, 2)[0]))
    start = err(amp(phi))
    assert exact < 0.15 * start
    assert compressed > 0.3 * start and compressed > 3 * exact
