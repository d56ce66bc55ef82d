"""Physical-space optimization through the library against the oracle (Sec. 3.2).

Deterministic parts (operator application, the TT of a combination) are
compared on amplitudes from random starts (unique truncations, as in
test_gpu_replica.py: 1e-9 of the largest amplitude per rounding chain).  The
sampled parts (H~, S~ by dual Monte Carlo) are compared with their exact
enumeration within a multiple of the reported standard errors.
"""
import numpy as np
import pytest

from paper_2604_22718_gb300 import inputs
from oracle import dual
from oracle import replica as rp

torch = pytest.importorskip("torch")

LX, LY, ORDER = 3, 2, ("H", "V")


def _operators():
    return [("1", []),
            ("X", inputs.replica_terms(LX, LY, ORDER, [], 1.0)),
            ("ZZ_HV", inputs.replica_terms(LX, LY, ORDER, [("H", 1.0, "H"), ("V", 1.0, "V")], 0.0))]


def _path():
    return inputs.path_sum([inputs.ordering(o, LX, LY) for o in ORDER])


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _opt(chi):
    from paper_2604_22718_gb300.physical import PhysicalOptimizer
    return PhysicalOptimizer(LX * LY, _path(), inputs.open_bonds(LX, LY), 1.0, 3.0, chi, _operators())


@pytest.mark.gpu
@pytest.mark.parametrize("chi", [2, 3])
def test_operator_states_match_oracle(chi):
    opt = _opt(chi)
    phi0 = inputs.replica_start(40 + chi, 12, chi)
    phis, logn = opt.operator_states(_dev(phi0))
    torch.cuda.synchronize()
    assert opt.chi_s == 2 * chi
    path = _path()
    for a, (_, terms) in enumerate(_operators()):
        if terms:
            eta, ops = rp.lift(terms, path, LX * LY)
        else:
            eta, ops = np.ones(1), np.zeros((1, path.shape[0]), dtype=np.uint8)
        assert tuple(phis[a].shape) == (12, 2, 2 * chi, 2 * chi)
        ref, nrm = rp.apply_operator(rp.unpadded(phi0), eta, ops, 2 * chi, chi_tree=4 * chi)
        got = rp.unpadded(phis[a].cpu().numpy())
        x, y = rp.tt_dense(got), rp.tt_dense(ref)
        assert np.abs(x - y).max() <= 1e-9 * np.abs(y).max()
        assert float(logn[a]) == pytest.approx(np.log(nrm), rel=1e-10, abs=1e-10)
    opt.close()


@pytest.mark.gpu
def test_sum_round_matches_oracle_combine():
    rtt = pytest.importorskip("paper_2604_22718_gb300.rtt")
    L, chi = 30, 2
    phis = [inputs.replica_start(70 + m, L, chi) for m in range(5)]
    c = np.array([0.5, -1.5, 2.0, 0.25, -0.75])
    plan = rtt.TTPlan(L, chi, np.ones(5), np.zeros((5, L), dtype=np.uint8))
    out = torch.empty((L, 2, chi, chi), dtype=torch.float64, device="cuda")
    ln = torch.empty(1, dtype=torch.float64, device="cuda")
    plan.sum_round([_dev(p) for p in phis], c, out, ln)
    torch.cuda.synchronize()
    ref, nrm = rp.combine([rp.unpadded(p) for p in phis], c, chi)
    rng = np.random.default_rng(1)
    idx = rng.integers(0, 2, size=(512, L))
    x, y = rp.tt_eval(rp.unpadded(out.cpu().numpy()), idx), rp.tt_eval(ref, idx)
    assert np.abs(x - y).max() <= 1e-9 * np.abs(y).max()
    assert float(ln.item()) == pytest.approx(np.log(nrm), rel=1e-10)
    with pytest.raises(rtt.RTTError, match="n exceeds"):
        plan.sum_round([_dev(p) for p in phis] + [_dev(phis[0])], np.ones(6), out)


@pytest.mark.gpu
def test_sum_round_and_apply_across_ranks():
    """Inputs of another rank than the plan's chi: rank-4 TTs summed with the
    tree at rank 4 and compressed to 2 (the physical-space combination), and a
    rank-2 TT put through a rank-4 plan (the operator states); a rank above
    max(chi, chi_tree) is rejected."""
    rtt = pytest.importorskip("paper_2604_22718_gb300.rtt")
    L = 24
    phis = [inputs.replica_start(90 + m, L, 4) for m in range(3)]
    c = np.array([1.0, -0.5, 0.75])
    plan = rtt.TTPlan(L, 2, np.ones(3), np.zeros((3, L), dtype=np.uint8), chi_tree=4)
    out = torch.empty((L, 2, 2, 2), dtype=torch.float64, device="cuda")
    ln = torch.empty(1, dtype=torch.float64, device="cuda")
    plan.sum_round([_dev(p) for p in phis], c, out, ln)
    torch.cuda.synchronize()
    ref, nrm = rp.combine([rp.unpadded(p) for p in phis], c, 2, chi_tree=4)
    idx = np.random.default_rng(2).integers(0, 2, size=(512, L))
    x, y = rp.tt_eval(rp.unpadded(out.cpu().numpy()), idx), rp.tt_eval(ref, idx)
    assert np.abs(x - y).max() <= 1e-9 * np.abs(y).max()
    assert float(ln.item()) == pytest.approx(np.log(nrm), rel=1e-10)
    with pytest.raises(rtt.RTTError, match="chi_in"):
        plan.sum_round([_dev(inputs.replica_start(95, L, 8))] * 2, np.ones(2), out)

    terms = inputs.replica_terms(LX, LY, ORDER, [("H", 0.7, "H"), ("V", -1.1, "V")], 2.0)
    path = _path()
    eta, ops = rp.lift(terms, path, LX * LY)
    up = rtt.TTPlan(12, 4, eta, ops, chi_tree=8)
    phi2 = inputs.replica_start(96, 12, 2)
    o4 = torch.empty((12, 2, 4, 4), dtype=torch.float64, device="cuda")
    ln4 = torch.empty(1, dtype=torch.float64, device="cuda")
    up.apply(_dev(phi2), o4, ln4)
    torch.cuda.synchronize()
    ref, nrm = rp.apply_operator(rp.unpadded(phi2), eta, ops, 4, chi_tree=8)
    x, y = rp.tt_dense(rp.unpadded(o4.cpu().numpy())), rp.tt_dense(ref)
    assert np.abs(x - y).max() <= 1e-9 * np.abs(y).max()
    assert float(ln4.item()) == pytest.approx(np.log(nrm), rel=1e-10)
    with pytest.raises(rtt.RTTError, match="chi_phi"):
        up.apply(_dev(inputs.replica_start(97, 12, 16)), o4)
    plan.close()
    up.close()


def _oracle_states(phi0, chi_s):
    """The operator states by the oracle alone, from the seeded start: its own
    lifting and apply_operator at rank chi_s (tree rank 2 chi_s), as RTT
    descriptions with b_L = b_R = e_0."""
    path = _path()
    e0v = np.zeros(chi_s)
    e0v[0] = 1.0
    out = []
    for _, terms in _operators():
        if terms:
            eta, ops = rp.lift(terms, path, LX * LY)
        else:
            eta, ops = np.ones(1), np.zeros((1, path.shape[0]), dtype=np.uint8)
        phi, _ = rp.apply_operator(rp.unpadded(phi0), eta, ops, chi_s, chi_tree=2 * chi_s)
        out.append(inputs.RTTInstance(n_spins=LX * LY, path=path.astype(np.int32),
                                      tensors=rp.padded(phi, chi_s), b_left=e0v, b_right=e0v.copy(),
                                      bonds=inputs.open_bonds(LX, LY), J=1.0, h=3.0))
    return out


@pytest.mark.gpu
def test_physical_step_against_exact_enumeration():
    """One iteration on 3x2 (four sites per spin pair, N = 6): sampled H~, S~
    within 6 standard errors (plus 1e-9) of their enumeration over the oracle's
    own operator states (built from the same seeded start); lambda_0 close to
    the exact one, which lies between the ground-state energy and the starting
    energy; the optimizer's combination of its states with fixed coefficients
    equal to the oracle's combination of its states; the step's TT that
    combination taken with the step's own c."""
    opt = _opt(2)
    phi0 = inputs.replica_start(77, 12, 2)
    spins0 = inputs.initial_spins(5, 4096, 6)
    res = opt.step(_dev(phi0), spins0, chains=4096, sweeps=200, burn=20, seed=31)
    torch.cuda.synchronize()
    states = _oracle_states(phi0, opt.chi_s)
    Ht, St = dual.exact_tilde_matrices(states)
    assert np.all(np.abs(res["Ht"] - Ht) <= 6 * res["Ht_se"] + 1e-9), (res["Ht"], Ht, res["Ht_se"])
    assert np.all(np.abs(res["St"] - St) <= 6 * res["St_se"] + 1e-9), (res["St"], St, res["St_se"])
    w, _ = dual.solve(Ht, St)
    lam = res["lambda"][0].real
    assert lam == pytest.approx(w[0].real, abs=0.02 * abs(w[0].real))
    # exact bounds: ground state <= lambda_0 (exact) <= energy of the start (identity included)
    H = _dense_tfim(6, inputs.open_bonds(LX, LY), 1.0, 3.0)
    path = _path()
    psi1 = rp.constrained_amplitudes(rp.unpadded(phi0), path, 6)
    assert np.linalg.eigvalsh(H)[0] - 1e-9 <= w[0].real <= psi1 @ H @ psi1 / (psi1 @ psi1) + 1e-9
    # the combination: fixed coefficients on both sides
    c = np.array([1.0, -0.35, 0.6])
    got = opt.combine(res["phis"], c)
    ref, _ = rp.combine([rp.unpadded(st.tensors) for st in states], c, 2)
    x, y = rp.tt_dense(rp.unpadded(got.cpu().numpy())), rp.tt_dense(ref)
    assert np.abs(x - y).max() <= 1e-9 * np.abs(y).max()
    again = opt.combine(res["phis"], res["c"])
    assert torch.equal(again, res["phi"])
    opt.close()


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["first", "all"])
def test_gram_schmidt_step_against_exact_enumeration(mode):
    """The iteration with Eq. Gram-Schmid: the pilot's S~ entries within 6
    standard errors of their enumeration over the oracle's states; T built from
    them (1 on the diagonal, -S~_am below it, column 0 only for 'first');
    lambda_0 from the Gram-Schmidt basis close to the exact one of the original
    basis (the basis does not change the eigenvalues); for 'first' the main
    pass's S~ against psi^1 near zero; c = T^T c' with c' from the library's
    solver."""
    rtt = pytest.importorskip("paper_2604_22718_gb300.rtt")
    opt = _opt(2)
    phi0 = inputs.replica_start(77, 12, 2)
    res = opt.step(_dev(phi0), inputs.initial_spins(5, 4096, 6), chains=4096, sweeps=200, burn=20,
                   seed=31, gram_schmidt=mode)
    torch.cuda.synchronize()
    T, P, Pse = res["T"], res["pilot_St"], res["pilot_St_se"]
    M = T.shape[0]
    Ht_x, St_x = dual.exact_tilde_matrices(_oracle_states(phi0, opt.chi_s))
    rows = [0] if mode == "first" else range(M)
    for a in rows:
        for m in range(M):
            assert abs(P[a, m] - St_x[a, m]) <= 6 * Pse[a, m] + 1e-9, (a, m, P, St_x, Pse)
    for m in range(M):
        for a in range(M):
            want = 1.0 if a == m else (-P[a, m] if a < m and (mode == "all" or a == 0) else 0.0)
            assert T[m, a] == want
    w_x, _ = dual.solve(Ht_x, St_x)
    assert res["lambda"][0].real == pytest.approx(w_x[0].real, abs=0.02 * abs(w_x[0].real))
    if mode == "first":
        for m in range(1, M):
            assert abs(res["St"][0, m]) <= 0.2 * abs(St_x[0, m]) + 15 * res["St_se"][0, m]
    _, cp = rtt.dual_solve(res["Ht"], res["St"])
    np.testing.assert_array_equal(res["c"], rtt.dual_back_transform(T, cp))
    np.testing.assert_allclose(res["c"], T.T @ cp, rtol=1e-13, atol=1e-13 * np.abs(cp).max())
    with pytest.raises(ValueError):
        opt.step(_dev(phi0), inputs.initial_spins(5, 64, 6), chains=64, sweeps=2, burn=1, seed=1,
                 gram_schmidt="second")
    opt.close()


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


@pytest.mark.gpu
def test_identity_only_iteration_keeps_the_state():
    """M = 1 (the identity): H~ = <E_loc>, S~ = 1, c = (1); the combined TT is
    the start itself (up to the unit-norm scaling)."""
    from paper_2604_22718_gb300.physical import PhysicalOptimizer
    opt = PhysicalOptimizer(LX * LY, _path(), inputs.open_bonds(LX, LY), 1.0, 3.0, 2, [("1", [])])
    phi0 = inputs.replica_start(78, 12, 2)
    res = opt.step(_dev(phi0), inputs.initial_spins(6, 1024, 6), chains=1024, sweeps=20, burn=5, seed=3)
    torch.cuda.synchronize()
    assert res["c"].shape == (1,) and res["c"][0] == pytest.approx(1.0)
    assert res["St"][0, 0] == pytest.approx(1.0, abs=1e-12)
    want = rp.tt_dense(rp.unpadded(phi0))
    got = rp.tt_dense(rp.unpadded(res["phi"].cpu().numpy()))
    np.testing.assert_allclose(got * np.linalg.norm(want), want, atol=1e-10 * np.abs(want).max())
    opt.close()
