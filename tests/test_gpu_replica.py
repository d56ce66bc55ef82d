"""Replica-space optimization through the C ABI against the oracle (Sec. 3.1).

Host lifting (no GPU) is compared bit for bit.  TT roundings and (1 - tau
H-bar) steps are compared on what is unique about a TT -- its amplitudes --
since the cores themselves are fixed only up to gauge.  Tolerance: both sides
run backward-stable FP64 factorizations (Householder QR, Jacobi or LAPACK
SVD), so one rounding agrees to a few hundred ulps of the largest amplitude;
a truncation amplifies that by 1 / (relative gap between the kept and the
dropped singular values), which the random inputs here keep far from zero.
1e-9 of the largest amplitude per rounding, 1e-7 after several steps.
"""
import numpy as np
import pytest

from paper_2604_22718_gb300 import inputs
from oracle import replica as rp

torch = pytest.importorskip("torch")


def _rtt():
    from paper_2604_22718_gb300 import rtt
    return rtt


# ---------------------------------------------------------------- host lifting (no GPU)

@pytest.mark.parametrize("kind", ["H", "HV", "HVDDp"])
@pytest.mark.parametrize("lx,ly", [(2, 3), (6, 6)])
def test_lift_matches_oracle_bitwise(kind, lx, ly):
    rtt = _rtt()
    order = ("V", "H", "D", "Dp")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    terms = inputs.hbar_terms(kind, lx, ly, 3.0, orderings=order)
    eta, ops = rtt.replica_lift(lx * ly, path, terms)
    e2, o2 = rp.lift(terms, path, lx * ly)
    assert np.array_equal(ops, o2) and np.array_equal(eta, e2)


def test_lift_rejects_bad_input():
    rtt = _rtt()
    path = inputs.path_sum([inputs.ordering(o, 2, 2) for o in ("H", "V")])
    with pytest.raises(rtt.RTTError, match="UNSUPPORTED"):
        rtt.replica_lift(4, path, [(1.0, [(0, "Y")], 0)])
    with pytest.raises(rtt.RTTError, match="twice"):
        rtt.replica_lift(4, path, [(1.0, [(1, "Z"), (1, "X")], 0)])
    with pytest.raises(rtt.RTTError, match="permutation"):
        rtt.replica_lift(4, np.asarray([0, 1, 2, 2, 0, 1, 2, 3]), [(1.0, [(0, "Z")], 0)])
    with pytest.raises(rtt.RTTError, match="block"):
        rtt.replica_lift(4, path, [(1.0, [(0, "Z")], 2)])


# ---------------------------------------------------------------- device helpers

def _dense_tfim(n, bonds, J, h):
    """H = J sum Z_i Z_j - h sum X_i by Kronecker products, spin 0 the MSB."""
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


def _dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _host_tt(cores_dev):
    return rp.unpadded(cores_dev.cpu().numpy())


def _compare(tt_gpu, tt_ref, L, tol, rng):
    """Dense amplitudes (L <= 14) or amplitudes at 512 random replica
    configurations, relative to the largest magnitude."""
    if L <= 14:
        a, b = rp.tt_dense(tt_gpu), rp.tt_dense(tt_ref)
    else:
        idx = rng.integers(0, 2, size=(512, L))
        a, b = rp.tt_eval(tt_gpu, idx), rp.tt_eval(tt_ref, idx)
    scale = np.abs(b).max()
    assert scale > 0
    err = np.abs(a - b).max() / scale
    assert err <= tol, f"max relative deviation {err:.3e}"


def _right_orthonormal(tt):
    for G in tt[1:]:
        M = G.reshape(G.shape[0], -1)
        gram = M @ M.T
        nz = np.abs(np.diag(gram)) > 0.5      # rows of rank-deficient bonds are zero
        np.testing.assert_allclose(gram[np.ix_(nz, nz)], np.eye(int(nz.sum())), atol=1e-12)


# ---------------------------------------------------------------- one rounding

@pytest.mark.gpu
@pytest.mark.parametrize("L,chi", [(2, 1), (2, 2), (3, 2), (7, 3), (12, 2), (12, 4), (37, 2),
                                   (37, 8), (64, 16), (144, 2)])
def test_round_sum_matches_oracle(L, chi):
    rtt = _rtt()
    rng = np.random.default_rng(1000 + 7 * L + chi)
    a = inputs.replica_start(11 + L, L, chi)
    b = inputs.replica_start(12 + L, L, chi)
    ops_a = rng.integers(0, 3, size=L).astype(np.uint8)
    ops_b = rng.integers(0, 3, size=L).astype(np.uint8)
    ca, cb = 0.8, -1.3
    plan = rtt.TTPlan(L, chi, np.ones(1), np.zeros((1, L), dtype=np.uint8))
    out = torch.empty((L, 2, chi, chi), dtype=torch.float64, device="cuda")
    plan.round_sum(_dev(a), _dev(b), out, ca, cb, _dev(ops_a, torch.uint8), _dev(ops_b, torch.uint8))
    torch.cuda.synchronize()
    ref = rp.tt_round(rp.tt_sum(rp.apply_string(rp.unpadded(a), ops_a, ca),
                                rp.apply_string(rp.unpadded(b), ops_b, cb)), chi)
    got = _host_tt(out)
    _compare(got, ref, L, 1e-9, rng)
    _right_orthonormal(got)


@pytest.mark.gpu
def test_round_sum_without_truncation_is_exact_and_normalises():
    """chi large enough for the sum: the rounding reproduces the sum itself."""
    rtt = _rtt()
    L, chi = 8, 8
    rng = np.random.default_rng(3)
    a = rp.padded(rp.tt_random(rng, L, 4), chi)
    b = rp.padded(rp.tt_random(rng, L, 4), chi)
    plan = rtt.TTPlan(L, chi, np.ones(1), np.zeros((1, L), dtype=np.uint8))
    out = torch.empty((L, 2, chi, chi), dtype=torch.float64, device="cuda")
    ln = torch.empty(1, dtype=torch.float64, device="cuda")
    plan.round_sum(_dev(a), _dev(b), out, 1.0, 2.0, log_norm=ln)
    torch.cuda.synchronize()
    want = rp.tt_dense(rp.unpadded(a)) + 2.0 * rp.tt_dense(rp.unpadded(b))
    got = rp.tt_dense(_host_tt(out))
    assert float(ln.item()) == pytest.approx(np.log(np.linalg.norm(want)), rel=1e-12)
    np.testing.assert_allclose(got * np.linalg.norm(want), want, atol=1e-12 * np.abs(want).max())
    assert np.linalg.norm(got) == pytest.approx(1.0, rel=1e-12)


@pytest.mark.gpu
def test_round_sum_of_a_tt_with_itself_and_of_zero():
    """Degenerate sums: a + a has the rank of a (many zero singular values);
    a - a is the zero TT."""
    rtt = _rtt()
    L, chi = 10, 2
    a = inputs.replica_start(5, L, chi)
    plan = rtt.TTPlan(L, chi, np.ones(1), np.zeros((1, L), dtype=np.uint8))
    out = torch.empty((L, 2, chi, chi), dtype=torch.float64, device="cuda")
    plan.round_sum(_dev(a), _dev(a), out, 1.0, 1.0)
    torch.cuda.synchronize()
    want = 2.0 * rp.tt_dense(rp.unpadded(a))
    np.testing.assert_allclose(rp.tt_dense(_host_tt(out)), want, atol=1e-12 * np.abs(want).max())
    plan.round_sum(_dev(a), _dev(a), out, 1.0, -1.0)
    torch.cuda.synchronize()
    assert np.abs(rp.tt_dense(_host_tt(out))).max() <= 1e-14 * np.abs(want).max()


# ---------------------------------------------------------------- (1 - tau H-bar) steps

def _power_case(lx, ly, order, kind, chi, steps, start, tau=0.1, h=3.0, seed=0, chi_tree=None):
    rtt = _rtt()
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    L = path.shape[0]
    terms = inputs.hbar_terms(kind, lx, ly, h, orderings=order)
    eta, ops = rtt.replica_lift(lx * ly, path, terms)
    eta_o, ops_o = rp.lift(terms, path, lx * ly)          # the oracle lifts on its own
    phi0 = inputs.replica_ones(L, chi) if start == "ones" else inputs.replica_start(seed, L, chi)
    ct = min(rp.tree_rank(chi, chi_tree), 16)
    plan = rtt.TTPlan(L, chi, eta, ops, chi_tree=ct)
    phi = _dev(phi0)
    ln = torch.empty(steps, dtype=torch.float64, device="cuda")
    plan.power(phi, tau, steps, log_norm=ln)
    torch.cuda.synchronize()
    ref, ref_ln = rp.power(rp.unpadded(phi0), eta_o, ops_o, tau, chi, steps, chi_tree=ct)
    return path, _host_tt(phi), ref, ln.cpu().numpy(), ref_ln


@pytest.mark.gpu
@pytest.mark.parametrize("lx,ly,order,kind,chi,steps,start", [
    (3, 2, ("H", "V"), "HV", 2, 5, "random"),      # L = 12, K = 13 (odd)
    (3, 2, ("H", "V"), "H", 4, 3, "random"),
    (2, 2, ("H", "V"), "HV", 16, 4, "ones"),       # no truncation
    (3, 3, ("V", "H", "D", "Dp"), "HVDDp", 2, 4, "random"),   # L = 36, K = 29
])
def test_power_steps_match_oracle(lx, ly, order, kind, chi, steps, start):
    path, got, ref, ln, ref_ln = _power_case(lx, ly, order, kind, chi, steps, start, seed=lx * 10 + chi)
    rng = np.random.default_rng(9)
    _compare(got, ref, len(path), 1e-7, rng)
    np.testing.assert_allclose(ln, ref_ln, rtol=1e-9, atol=1e-9)
    assert rp.tt_norm(got) == pytest.approx(1.0, rel=1e-10)


@pytest.mark.gpu
@pytest.mark.parametrize("chi,chi_tree", [(2, 2), (2, 3), (3, 6)])
def test_power_steps_with_other_tree_ranks(chi, chi_tree):
    """The tree's pairwise sums rounded to chi_tree (chi itself: every sum
    truncated to the final rank; between chi and 2 chi)."""
    path, got, ref, ln, ref_ln = _power_case(3, 2, ("H", "V"), "HV", chi, 4, "random", seed=90 + chi,
                                            chi_tree=chi_tree)
    _compare(got, ref, len(path), 1e-7, np.random.default_rng(4))
    np.testing.assert_allclose(ln, ref_ln, rtol=1e-9, atol=1e-9)


@pytest.mark.gpu
def test_power_steps_6x6_workload_sampled():
    """The 6x6 workload's shapes (path V+H+D+D', L = 144, 96 terms, chi = 2),
    three steps from a random TT, amplitudes at sampled configurations."""
    path, got, ref, ln, ref_ln = _power_case(6, 6, ("V", "H", "D", "Dp"), "HV", 2, 3, "random",
                                            seed=66)
    rng = np.random.default_rng(10)
    _compare(got, ref, len(path), 1e-7, rng)
    np.testing.assert_allclose(ln, ref_ln, rtol=1e-9, atol=1e-9)


@pytest.mark.gpu
def test_power_single_term_and_two_terms():
    """K = 1 (no tree: phi - tau eta P phi) and K = 2 (one tree level)."""
    rtt = _rtt()
    L, chi = 9, 3
    rng = np.random.default_rng(21)
    for K in (1, 2):
        ops = rng.integers(0, 3, size=(K, L)).astype(np.uint8)
        eta = rng.uniform(-2, 2, size=K)
        phi0 = inputs.replica_start(30 + K, L, chi)
        plan = rtt.TTPlan(L, chi, eta, ops)
        phi = _dev(phi0)
        plan.power(phi, 0.2, 2)
        torch.cuda.synchronize()
        ref, _ = rp.power(rp.unpadded(phi0), eta, ops, 0.2, chi, 2)
        _compare(_host_tt(phi), ref, L, 1e-8, rng)


@pytest.mark.gpu
def test_power_result_feeds_the_sampler():
    """phi^(P) as an RTT handle (b_L = b_R = e_0, same path): the sampler's
    amplitudes are C phi^(P) of the same cores (the oracle's phi^(P), so that
    the expected amplitudes come from the oracle alone)."""
    rtt = _rtt()
    lx, ly, chi = 3, 3, 2
    order = ("V", "H", "D", "Dp")
    path, _, got, _, _ = _power_case(lx, ly, order, "HV", chi, 6, "random", seed=8)
    e0 = np.zeros(chi)
    e0[0] = 1.0
    inst = inputs.RTTInstance(n_spins=9, path=path.astype(np.int32), tensors=rp.padded(got, chi),
                              b_left=e0, b_right=e0.copy(), bonds=inputs.open_bonds(lx, ly),
                              J=1.0, h=3.0)
    h = rtt.RTT(inst, precision="fp64")
    spins = inputs.initial_spins(4, 256, 9)
    log_abs, sign, _ = h.log_amplitudes(_dev(spins, torch.uint8))
    amp = sign.cpu().numpy() * np.exp(log_abs.cpu().numpy())
    want = rp.tt_eval(got, spins[:, path])
    np.testing.assert_allclose(amp, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())


@pytest.mark.gpu
def test_symmetric_start_energy_is_valid():
    """From phi^(0) = 1 (the paper's start) the lattice symmetry makes singular
    values at the cut exactly degenerate, so the rank-chi truncation is not
    unique: the kernel's Jacobi SVD and the oracle's LAPACK SVD keep different,
    equally valid subspaces and the trajectories differ.  What both must share:
    the energy of psi = C phi (exact, by enumeration) lies above the ground
    state, and the two energy errors agree to within a quarter of each other."""
    lx, ly, chi = 3, 3, 2
    order = ("V", "H", "D", "Dp")
    path, got, ref, ln, ref_ln = _power_case(lx, ly, order, "HV", chi, 6, "ones")
    H = _dense_tfim(9, inputs.open_bonds(lx, ly), 1.0, 3.0)
    e0 = np.linalg.eigvalsh(H)[0]

    def err(tt):
        psi = rp.constrained_amplitudes(tt, path, 9)
        return (psi @ H @ psi / (psi @ psi) - e0) / abs(e0)
    eg, eo = err(got), err(ref)
    assert eg >= -1e-12 and eo >= -1e-12
    assert abs(eg - eo) <= 0.25 * eo, (eg, eo)
    assert eg < 0.03                     # well below the start's 3.8 %
    assert np.all(np.isfinite(ln))


@pytest.mark.gpu
def test_plan_rejects_bad_arguments():
    rtt = _rtt()
    with pytest.raises(rtt.RTTError, match="UNSUPPORTED"):
        rtt.TTPlan(8, 17, np.ones(1), np.zeros((1, 8), dtype=np.uint8))
    with pytest.raises(rtt.RTTError, match="INVALID_ARG"):
        rtt.TTPlan(1, 2, np.ones(1), np.zeros((1, 1), dtype=np.uint8))
    with pytest.raises(rtt.RTTError, match="INVALID_ARG"):
        rtt.TTPlan(8, 2, np.ones(1), np.full((1, 8), 3, dtype=np.uint8))
    with pytest.raises(rtt.RTTError, match="INVALID_ARG"):
        rtt.TTPlan(8, 2, np.ones(0), np.zeros((0, 8), dtype=np.uint8))
    with pytest.raises(rtt.RTTError, match="chi_tree"):
        rtt.TTPlan(8, 4, np.ones(1), np.zeros((1, 8), dtype=np.uint8), chi_tree=3)
    plan = rtt.TTPlan(8, 2, np.ones(1), np.zeros((1, 8), dtype=np.uint8))
    a = torch.zeros((8, 2, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(rtt.RTTError, match="alias"):
        plan.round_sum(a, a, a)
    # zero steps leave phi untouched
    phi = _dev(inputs.replica_start(3, 8, 2))
    before = phi.clone()
    plan.power(phi, 0.1, 0)
    torch.cuda.synchronize()
    assert torch.equal(phi, before)


# ---------------------------------------------------------------- FP32 arithmetic

def _min_gap(tt, chi):
    """Smallest relative gap (sigma_chi - sigma_chi+1) / sigma_chi over the
    truncated bonds of the oracle's own rounding of tt."""
    L = len(tt)
    cores = [G.copy() for G in tt]
    for k in range(L - 1):
        r0, _, r1 = cores[k].shape
        Q, R = np.linalg.qr(cores[k].reshape(r0 * 2, r1))
        cores[k] = Q.reshape(r0, 2, -1)
        cores[k + 1] = np.einsum("ab,bsc->asc", R, cores[k + 1])
    gap = 1.0
    for k in range(L - 1, 0, -1):
        r0, _, r1 = cores[k].shape
        U, S, Vt = np.linalg.svd(cores[k].reshape(r0, 2 * r1), full_matrices=False)
        if len(S) > chi and S[chi - 1] > 1e-12 * S[0]:
            gap = min(gap, (S[chi - 1] - S[chi]) / S[chi - 1])
        t = min(chi, len(S))
        cores[k] = Vt[:t].reshape(t, 2, r1)
        cores[k - 1] = np.einsum("asb,bc->asc", cores[k - 1], U[:, :t] * S[:t])
    return gap


@pytest.mark.gpu
@pytest.mark.parametrize("L,chi", [(2, 1), (3, 2), (12, 2), (37, 2), (37, 8), (64, 16), (144, 2)])
def test_round_sum_fp32_within_derived_tolerance(L, chi):
    """FP32 roundings: 2L factorizations, each backward stable to a small
    multiple of u = 2^-24 relative, the truncations amplifying by 1/gap:
    tolerance 16 u 2L / gap of the largest amplitude (gap from the oracle)."""
    rtt = _rtt()
    rng = np.random.default_rng(2000 + 7 * L + chi)
    a = inputs.replica_start(11 + L, L, chi)
    b = inputs.replica_start(12 + L, L, chi)
    ops_a = rng.integers(0, 3, size=L).astype(np.uint8)
    ops_b = rng.integers(0, 3, size=L).astype(np.uint8)
    s = rp.tt_sum(rp.apply_string(rp.unpadded(a), ops_a, 0.8),
                  rp.apply_string(rp.unpadded(b), ops_b, -1.3))
    ref = rp.tt_round(s, chi)
    tol = 16 * 2.0 ** -24 * 2 * L / _min_gap(s, chi)
    plan = rtt.TTPlan(L, chi, np.ones(1), np.zeros((1, L), dtype=np.uint8), precision="fp32")
    out = torch.empty((L, 2, chi, chi), dtype=torch.float64, device="cuda")
    plan.round_sum(_dev(a), _dev(b), out, 0.8, -1.3, _dev(ops_a, torch.uint8), _dev(ops_b, torch.uint8))
    torch.cuda.synchronize()
    _compare(_host_tt(out), ref, L, tol, rng)


def _oracle_power_with_gaps(phi, eta, ops, tau, chi, steps):
    """The oracle's steps (same tree, same roundings) and the smallest
    truncation gap met by any rounding on the way."""
    gap = 1.0
    ct = rp.tree_rank(chi)
    for _ in range(steps):
        items = [rp.apply_string(phi, ops[k], eta[k]) for k in range(len(eta))]
        while len(items) > 1:
            nxt = []
            for i in range(0, len(items) - 1, 2):
                s = rp.tt_sum(items[i], items[i + 1])
                gap = min(gap, _min_gap(s, ct))
                nxt.append(rp.tt_round(s, ct))
            if len(items) % 2:
                nxt.append(items[-1])
            items = nxt
        s = rp.tt_sum(phi, rp.tt_scale(items[0], -tau))
        gap = min(gap, _min_gap(s, chi))
        phi = rp.tt_scale(rp.tt_round(s, chi), 1.0)
        phi = rp.tt_scale(phi, 1.0 / rp.tt_norm(phi))
    return phi, gap


@pytest.mark.gpu
def test_power_fp32_amplitudes_within_derived_tolerance():
    """One FP32 (1 - tau H-bar) step from a random start on 3x3 (path
    V+H+D+D', chi = 2, 21 terms: 5 tree levels + the final rounding): each of
    the 6 roundings in sequence contributes at most 16 u 2L / gap of the
    largest amplitude (u = 2^-24, gap = the smallest truncation gap the
    oracle's own run meets, 0.015 here).  Longer runs meet near-degenerate
    truncations (gap 4e-5 in the second step) where any two correct
    implementations may part; they are checked on the energy instead."""
    rtt = _rtt()
    lx = ly = 3
    order = ("V", "H", "D", "Dp")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    L = path.shape[0]
    terms = inputs.hbar_terms("HV", lx, ly, 3.0, orderings=order)
    eta, ops = rtt.replica_lift(9, path, terms)
    eta_o, ops_o = rp.lift(terms, path, 9)
    phi0 = inputs.replica_start(91, L, 2)
    plan = rtt.TTPlan(L, 2, eta, ops, precision="fp32")
    phi = _dev(phi0)
    steps = 1
    plan.power(phi, 0.1, steps)
    torch.cuda.synchronize()
    ref, gap = _oracle_power_with_gaps(rp.unpadded(phi0), eta_o, ops_o, 0.1, 2, steps)
    tol = 16 * 2.0 ** -24 * 2 * L * steps * 6 / gap
    _compare(_host_tt(phi), ref, L, tol, np.random.default_rng(12))


@pytest.mark.gpu
def test_power_fp32_symmetric_start_energy_is_valid():
    """From phi^(0) = 1 the first truncations are degenerate (equal singular
    values at the cut, so the kept subspace is not unique): the FP32 run's
    exact energy is variational and within a quarter of the oracle run's
    error."""
    rtt = _rtt()
    lx = ly = 3
    order = ("V", "H", "D", "Dp")
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    L = path.shape[0]
    terms = inputs.hbar_terms("HV", lx, ly, 3.0, orderings=order)
    eta, ops = rtt.replica_lift(9, path, terms)
    eta_o, ops_o = rp.lift(terms, path, 9)
    phi0 = inputs.replica_ones(L, 2)
    plan = rtt.TTPlan(L, 2, eta, ops, precision="fp32")
    phi = _dev(phi0)
    plan.power(phi, 0.1, 6)
    torch.cuda.synchronize()
    ref, _ = rp.power(rp.unpadded(phi0), eta_o, ops_o, 0.1, 2, 6)
    H = _dense_tfim(9, inputs.open_bonds(lx, ly), 1.0, 3.0)
    e0 = np.linalg.eigvalsh(H)[0]

    def energy(tt):
        psi = rp.constrained_amplitudes(tt, path, 9)
        return psi @ H @ psi / (psi @ psi)
    eg, eo = energy(_host_tt(phi)), energy(ref)
    assert eg >= e0 - 1e-9 and abs((eg - e0) - (eo - e0)) <= 0.25 * (eo - e0)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_round_sum_beyond_fp32_range(precision):
    """A TT whose norm overflows FP32 (every core of a random TT doubled on 144
    sites: 2^144 more) and whose first core is 2^100 larger still: the kernel
    carries the scale as a power-of-two exponent, so the rounding is finite,
    agrees with the oracle within the derived tolerance, and the log-norm
    carries the scale."""
    rtt = _rtt()
    L, chi = 144, 2
    rng = np.random.default_rng(31)
    a = inputs.replica_start(501, L, chi) * 2.0
    b = inputs.replica_start(502, L, chi) * 2.0
    a[0] *= 2.0 ** 100
    b[0] *= 2.0 ** 100
    s = rp.tt_sum(rp.unpadded(a), rp.unpadded(b))
    ref = rp.tt_round(s, chi)
    tol = 1e-9 if precision == "fp64" else 16 * 2.0 ** -24 * 2 * L / _min_gap(s, chi)
    plan = rtt.TTPlan(L, chi, np.ones(1), np.zeros((1, L), dtype=np.uint8), precision=precision)
    out = torch.empty((L, 2, chi, chi), dtype=torch.float64, device="cuda")
    ln = torch.empty(1, dtype=torch.float64, device="cuda")
    plan.round_sum(_dev(a), _dev(b), out, 1.0, 1.0, log_norm=ln)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    nrm = rp.tt_norm(ref)
    assert float(ln.item()) == pytest.approx(np.log(nrm), rel=1e-6 if precision == "fp32" else 1e-12)
    _compare(rp.tt_scale(rp.unpadded(got), nrm), ref, L, tol, rng)
