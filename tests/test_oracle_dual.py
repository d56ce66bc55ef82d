"""Pins of the dual Monte Carlo oracle (Sec. 3.3) against dense linear algebra.

Each check compares the oracle with something other than itself: a dense TFIM
matrix built from Kronecker products, exact amplitude vectors, the projected
symmetric eigenproblem (scipy), algebraic identities of the method.
"""
import numpy as np
import pytest

from paper_2604_22718_gb300 import inputs
from oracle import oracle as orc
from oracle import dual


def _dense_tfim(n, bonds, J, h):
    """H = J sum Z_i Z_j - h sum X_i, spin 0 the most significant bit, s = 0 <-> Z = +1."""
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


def _states(M, chi=3, seeds=(31, 32, 33, 34, 35), mixing=True, R=2):
    return [inputs.make_instance(3, 3, R, chi, 3.0, seed=s, mixing=mixing) for s in seeds[:M]]


def _psi_matrix(states):
    return np.stack([orc.Oracle(s).all_amplitudes() for s in states], axis=1)   # [2^N][M]


def test_mixed_local_energy_is_h_psi_b_over_psi_a():
    a, b = _states(2)
    H = _dense_tfim(9, a.bonds, a.J, a.h)
    pa, pb = orc.Oracle(a).all_amplitudes(), orc.Oracle(b).all_amplitudes()
    spins = dual.all_configurations(9)
    e, r = dual.mixed_local_energies(orc.Oracle(a), orc.Oracle(b), spins)
    want_e = (H @ pb) / pa
    scale = np.abs(want_e).max()
    assert np.max(np.abs(e - want_e)) <= 1e-11 * scale
    np.testing.assert_allclose(r, pb / pa, rtol=1e-12)


def test_same_state_gives_vmc_local_energy_and_unit_ratio():
    (a,) = _states(1)
    o = orc.Oracle(a)
    spins = inputs.initial_spins(3, 40, 9)
    e, r = dual.mixed_local_energies(o, o, spins)
    assert np.all(r == 1.0)
    np.testing.assert_allclose(e, o.local_energies(spins), rtol=1e-13, atol=1e-13)


def test_tilde_matrices_against_dense_projection():
    states = _states(3)
    Ht, St = dual.exact_tilde_matrices(states)
    H = _dense_tfim(9, states[0].bonds, states[0].J, states[0].h)
    P = _psi_matrix(states)
    Hd, Sd = P.T @ H @ P, P.T @ P
    Z = np.diag(Sd)
    np.testing.assert_allclose(Ht, Hd / Z[:, None], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(St, Sd / Z[:, None], rtol=1e-10, atol=1e-12)
    # identities of the method: S~_aa = 1, H~_aa = <H>_a, Z_a H~_ab = Z_b H~_ba
    np.testing.assert_allclose(np.diag(St), 1.0, rtol=1e-13)
    for k, s in enumerate(states):
        assert Ht[k, k] == pytest.approx(orc.Oracle(s).exact_energy(), rel=1e-10)
    Hsym = Z[:, None] * Ht
    np.testing.assert_allclose(Hsym, Hsym.T, rtol=1e-9)


def test_generalized_eigenvalues_equal_projected_problem_and_bound_ground_state():
    import scipy.linalg
    states = _states(3)
    Ht, St = dual.exact_tilde_matrices(states)
    w, c = dual.solve(Ht, St)
    H = _dense_tfim(9, states[0].bonds, states[0].J, states[0].h)
    P = _psi_matrix(states)
    want = scipy.linalg.eigh(P.T @ H @ P, P.T @ P, eigvals_only=True)
    np.testing.assert_allclose(np.sort(w.real), np.sort(want), rtol=1e-9)
    assert np.max(np.abs(w.imag)) < 1e-9 * np.max(np.abs(w.real))
    e0 = np.linalg.eigvalsh(H)[0]
    assert w.real[0] >= e0 - 1e-9
    assert w.real[0] <= min(Ht[k, k] for k in range(3)) + 1e-9   # the span contains each state
    # the eigenvector: residual and normalisation
    np.testing.assert_allclose(Ht @ c, w.real[0] * (St @ c), atol=1e-9 * np.abs(Ht).max())
    assert abs(c @ St @ c) == pytest.approx(1.0, rel=1e-12)
    # the Rayleigh quotient of psi' = sum c_a psi^a is lambda_0
    v = P @ c
    assert (v @ H @ v) / (v @ v) == pytest.approx(w.real[0], rel=1e-9)


def test_one_state_eigenvalue_is_its_energy():
    (a,) = _states(1)
    Ht, St = dual.exact_tilde_matrices([a])
    w, c = dual.solve(Ht, St)
    assert w.real[0] == pytest.approx(orc.Oracle(a).exact_energy(), rel=1e-12)
    assert c[0] == pytest.approx(1.0)


def test_direct_sum_amplitude_is_the_linear_combination():
    states = _states(3, chi=2, mixing=False)
    coef = np.array([0.7, -1.3, 2.1])
    s_sum = dual.direct_sum(states, coef)
    assert s_sum.tensors.shape[2] == 6
    got = orc.Oracle(s_sum).all_amplitudes()
    want = _psi_matrix(states) @ coef
    assert np.max(np.abs(got - want)) <= 1e-12 * np.abs(want).max()


def test_direct_sum_rejects_other_lattices():
    a = inputs.make_instance(3, 3, 2, 2, 3.0, seed=1)
    b = inputs.make_instance(3, 3, 2, 2, 3.1, seed=2)       # another field
    with pytest.raises(AssertionError):
        dual.direct_sum([a, b], [1.0, 1.0])


@pytest.mark.parametrize("first_only", [True, False])
def test_gram_schmidt_orthogonalises_against_first_state_and_keeps_eigenvalues(first_only):
    states = _states(3)
    Ht, St = dual.exact_tilde_matrices(states)
    T = dual.gram_schmidt(St, first_only=first_only)
    assert np.allclose(np.triu(T, 1), 0) and np.allclose(np.diag(T), 1)
    new = [dual.direct_sum(states, T[m]) for m in range(3)]
    Ht2, St2 = dual.exact_tilde_matrices(new)
    # linearity: <psi'^m / psi^1>_{P^1} = sum_g T_mg S~_1g for every m ...
    np.testing.assert_allclose(St2[0], T @ St[0], atol=1e-12)
    # ... which vanishes for the second state always and, against psi^1 only, for all
    np.testing.assert_allclose(St2[0, 1], 0.0, atol=1e-12)
    if first_only:
        np.testing.assert_allclose(St2[0, 1:], 0.0, atol=1e-12)
    w1, _ = dual.solve(Ht, St)
    w2, _ = dual.solve(Ht2, St2)
    np.testing.assert_allclose(np.sort(w2.real), np.sort(w1.real), rtol=1e-9)
