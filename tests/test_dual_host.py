"""rtt_dual_solve (host code of the C library, no GPU) against the oracle's
library eigen-solver, and argument errors of the dual Monte Carlo entry points."""
import ctypes

import numpy as np
import pytest

from paper_2604_22718_gb300 import build as rtt_build
from paper_2604_22718_gb300 import inputs
from oracle import dual


@pytest.fixture(scope="module")
def rtt():
    rtt_build.build()
    from paper_2604_22718_gb300 import rtt as mod
    return mod


def _states(M, chi=3):
    return [inputs.make_instance(3, 3, 2, chi, 3.0, seed=s, mixing=True) for s in (41, 42, 43, 44)[:M]]


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_solve_matches_oracle_on_exact_matrices(rtt, M):
    Ht, St = dual.exact_tilde_matrices(_states(M))
    w, c = rtt.dual_solve(Ht, St)
    w_o, c_o = dual.solve(Ht, St)
    np.testing.assert_allclose(w.real, w_o.real, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(w.imag, 0.0, atol=1e-9 * np.abs(w).max())
    np.testing.assert_allclose(c, c_o, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(Ht @ c, w.real[0] * (St @ c), atol=1e-8 * np.abs(Ht).max())


def test_solve_random_pencils_and_complex_pairs(rtt):
    rng = np.random.default_rng(5)
    for M in range(1, 9):
        for _ in range(5):
            Ht = rng.standard_normal((M, M))
            St = rng.standard_normal((M, M)) + M * np.eye(M)
            w, c = rtt.dual_solve(Ht, St)
            w_o, _ = dual.solve(Ht, St)
            scale = np.abs(w_o).max()
            # the same multiset (conjugate pairs may come in either order)
            left = list(w_o)
            for z in w:
                k = int(np.argmin([abs(z - y) for y in left]))
                assert abs(z - left.pop(k)) <= 1e-9 * scale, (w, w_o)
            assert np.all(np.diff(w.real) >= -1e-12 * scale)
            if abs(w[0].imag) <= 1e-9 * scale:
                np.testing.assert_allclose(Ht @ c, w.real[0] * (St @ c), atol=1e-7 * scale * M)
                assert abs(c @ St @ c) == pytest.approx(1.0, rel=1e-9)
            else:
                assert np.all(np.isnan(c))


def test_solve_rejects_singular_overlap_and_bad_sizes(rtt):
    with pytest.raises(rtt.RTTError):
        rtt.dual_solve(np.eye(2), np.zeros((2, 2)))
    with pytest.raises(rtt.RTTError):
        rtt.dual_solve(np.eye(9), np.eye(9))
    lib = rtt.lib()
    assert lib.rtt_dual_solve(0, None, None, None, None, None) == 1


def test_dual_entry_points_reject_null_arguments(rtt):
    lib = rtt.lib()
    assert lib.rtt_mixed_local_energy(None, None, None, 4, None, None, None) == 1
    out = ctypes.c_void_p()
    assert lib.rtt_create_sum(None, 2, None, ctypes.byref(out)) == 1


@pytest.mark.parametrize("first_only", [True, False])
def test_gram_schmidt_basis_matches_oracle_and_keeps_the_pencil(rtt, first_only):
    """The physical step's Gram-Schmidt basis T (Eq. Gram-Schmid) equals the
    oracle's; the eigenvalues of the pencil in that basis, (T H T^T, T S T^T)
    on the symmetric matrices H = Z H~, S = Z S~, are those of the original,
    and c = T^T c' maps its lowest eigenvector back."""
    from paper_2604_22718_gb300.physical import PhysicalOptimizer
    Ht, St = dual.exact_tilde_matrices(_states(4))
    T = PhysicalOptimizer.gram_schmidt_matrix(St, first_only)
    np.testing.assert_array_equal(T, dual.gram_schmidt(St, first_only=first_only))
    # Z_a from S~ (S_ab = Z_a S~_ab symmetric): Z_a / Z_0 = S~_0a / S~_a0
    Z = np.array([St[0, a] / St[a, 0] for a in range(4)])
    H, S = Z[:, None] * Ht, Z[:, None] * St
    w, _ = rtt.dual_solve(H, S)
    wp, cp = rtt.dual_solve(T @ H @ T.T, T @ S @ T.T)
    np.testing.assert_allclose(wp.real, w.real, rtol=1e-9, atol=1e-12)
    c = T.T @ cp
    np.testing.assert_allclose(H @ c, wp[0].real * (S @ c), atol=1e-9 * np.abs(H @ c).max())


def test_physical_optimizer_rejects_state_ranks_outside_chi_to_16(rtt):
    """The operator states' rank must lie in [chi, 16] (host check, before any
    device allocation)."""
    from paper_2604_22718_gb300.physical import PhysicalOptimizer
    path = inputs.path_sum([inputs.ordering(o, 3, 2) for o in ("H", "V")])
    ops = [("1", []), ("X", inputs.replica_terms(3, 2, ("H", "V"), [], 1.0))]
    for bad in (1, 17):
        with pytest.raises(ValueError, match="chi_states"):
            PhysicalOptimizer(6, path, inputs.open_bonds(3, 2), 1.0, 3.0, 2, ops, chi_states=bad)


def test_gram_schmidt_and_back_transform_host_calls(rtt):
    """rtt_dual_gram_schmidt writes the oracle's T bit for bit (only the S~
    entries it uses must be finite: row 0 for the first-only form);
    rtt_dual_back_transform is T^T c'; both reject bad sizes, null pointers
    and an aliased output."""
    Ht, St = dual.exact_tilde_matrices(_states(4))
    for first_only in (True, False):
        T = rtt.dual_gram_schmidt(St, first_only)
        np.testing.assert_array_equal(T, dual.gram_schmidt(St, first_only=first_only))
        cp = np.array([0.3, -1.1, 2.5, 0.75])
        np.testing.assert_allclose(rtt.dual_back_transform(T, cp), T.T @ cp, rtol=1e-15, atol=1e-15)
    row0 = np.full((4, 4), np.nan)
    row0[0] = St[0]
    np.testing.assert_array_equal(rtt.dual_gram_schmidt(row0, True), dual.gram_schmidt(St, True))
    with pytest.raises(rtt.RTTError):
        rtt.dual_gram_schmidt(row0, False)          # rows 1.. are used and not finite
    lib = rtt.lib()
    buf = np.zeros(81)
    assert lib.rtt_dual_gram_schmidt(0, buf.ctypes.data, 1, buf.ctypes.data) == 1
    assert lib.rtt_dual_gram_schmidt(9, buf.ctypes.data, 1, buf.ctypes.data) == 1
    assert lib.rtt_dual_gram_schmidt(2, None, 1, buf.ctypes.data) == 1
    v = np.ones(4)
    assert lib.rtt_dual_back_transform(4, buf.ctypes.data, v.ctypes.data, v.ctypes.data) == 1
    assert lib.rtt_dual_back_transform(4, None, v.ctypes.data, buf.ctypes.data) == 1


def test_gram_schmidt_error_leaves_the_output_untouched(rtt):
    """A non-finite S~ entry that T uses (here S~[1][2], found after row 0 has
    been read) is reported as RTT_ERR_NUMERIC before any entry of the
    caller's T is written."""
    _, St = dual.exact_tilde_matrices(_states(4))
    bad = St.copy()
    bad[1, 2] = np.nan
    T = np.full((4, 4), 7.25)
    st = rtt.lib().rtt_dual_gram_schmidt(4, np.ascontiguousarray(bad).ctypes.data, 0, T.ctypes.data)
    assert st == 4
    assert np.all(T == 7.25)
