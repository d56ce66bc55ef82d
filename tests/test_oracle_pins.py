"""Pins of the FP64 oracle against things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle (a transposed
operand, a dropped boundary vector, a wrong sign of h or J, a wrong replica
set, an off-by-one in the path or the flip segment, a wrong RNG round) fails
at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_22718_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _inst(path, chi, seed, n=None, bonds=None, J=1.0, h=3.0, tensors=None):
    path = np.asarray(path, dtype=np.int32)
    n = int(path.max()) + 1 if n is None else n
    rng = np.random.default_rng(seed)
    L = path.shape[0]
    t = rng.standard_normal((L, 2, chi, chi)) / np.sqrt(chi) if tensors is None else tensors
    return inputs.RTTInstance(n_spins=n, path=path, tensors=np.ascontiguousarray(t),
                              b_left=rng.standard_normal(chi), b_right=rng.standard_normal(chi),
                              bonds=np.zeros((0, 2), np.int32) if bonds is None else bonds,
                              J=J, h=h)


def _psi(o, s):
    m, e = o.amplitude(s)
    return math.ldexp(m, e)


def _dense_product(inst, s):
    """b_L^T A_0[s_p(0)] ... A_{L-1}[s_p(L-1)] b_R by numpy matmul (other order)."""
    mats = [inst.tensors[k, s[inst.path[k]]] for k in range(inst.path.shape[0])]
    return float(inst.b_left @ np.linalg.multi_dot(mats + [inst.b_right])) if len(mats) > 1 \
        else float(inst.b_left @ mats[0] @ inst.b_right)


def _all_spins(n):
    return np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)


# --------------------------------------------------------------------------- Philox

def _numpy_philox_block(counter, key):
    """numpy's Philox (4x64, 10 rounds) yields the block of counter+1 first."""
    c = [int(x) for x in counter]
    assert c[0] >= 1
    c[0] -= 1
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64),
                         key=np.array([int(k) for k in key], dtype=np.uint64))
    return bg.random_raw(4).astype(np.uint64)


@pytest.mark.parametrize("counter,key", [
    ([1, 0, 0, 0], [0, 0]),
    ([7, 3, 11, 0], [22718, 0x4D434D43]),
    ([2**63 + 5, 2**64 - 1, 12345678901234, 42], [2**64 - 2, 977]),
    ([99, 1999, 35, 0], [22720, 0x4D434D43]),
])
def test_philox4x64_matches_numpy(counter, key):
    ours = orc.philox4x64(counter, key)
    ref = _numpy_philox_block(counter, key)
    assert np.array_equal(ours, ref)


def test_mcmc_uniform_is_top_53_bits_of_first_word():
    for (seed, c, t, j) in [(1, 1, 0, 0), (22720, 4095, 1999, 35), (5, 17, 3, 8)]:
        x = _numpy_philox_block([c, t, j, 0], [seed, 0x4D434D43])
        u = float(int(x[0]) >> 11) * 2.0 ** -53
        assert orc.mcmc_uniform(seed, c, t, j) == u
        assert 0.0 <= u < 1.0


# --------------------------------------------------------------------------- amplitude

def test_amplitude_matches_dense_product():
    inst = _inst(np.tile(np.arange(5), 3), chi=6, seed=1)
    o = orc.Oracle(inst)
    rng = np.random.default_rng(2)
    for _ in range(20):
        s = rng.integers(0, 2, 5).astype(np.uint8)
        ref = _dense_product(inst, s)
        assert _psi(o, s) == pytest.approx(ref, rel=1e-12, abs=0)


def _load_paths():
    paths = {}
    with open(os.path.join(GOLDEN, "psi_hv_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, *idx = line.split()
            paths[name] = np.array([int(x) - 1 for x in idx], dtype=np.int32)
    return paths


def test_worked_example_paths_and_path_sum():
    """Sec. 2.2.1: sigma^HV = sigma^H (+) sigma^V and psi^HV is the printed product."""
    p = _load_paths()
    assert np.array_equal(p["HV"], np.concatenate([p["H"], p["V"]]))
    chi = 3
    inst = _inst(p["HV"], chi=chi, seed=3, n=6)
    o = orc.Oracle(inst)
    A = inst.tensors
    for s in _all_spins(6):
        s1, s2, s3, s4, s5, s6 = (int(x) for x in s)
        # the explicit twelve-factor product as printed, 1-based site labels
        seq = [(1, s1), (2, s2), (3, s3), (4, s4), (5, s5), (6, s6),
               (7, s4), (8, s3), (9, s2), (10, s5), (11, s6), (12, s1)]
        m = np.eye(chi)
        for site, spin in seq:
            m = m @ A[site - 1, spin]
        ref = float(inst.b_left @ m @ inst.b_right)
        assert _psi(o, s) == pytest.approx(ref, rel=1e-12, abs=1e-300)


def test_constraint_formulation_psi_equals_C_phi():
    """Sec. 2.2.3: psi = C phi, phi the plain TT over Omega replica indices and
    C the product of Kronecker deltas tying the indices of R_j to s_j."""
    p = _load_paths()["HV"]
    chi = 2
    inst = _inst(p, chi=chi, seed=4, n=6)
    o = orc.Oracle(inst)
    Om = p.shape[0]
    # phi over all 2^Omega replica configurations by dense contraction
    phi = np.einsum("a,iab->ib", inst.b_left, inst.tensors[0])   # [i1][b]
    for k in range(1, Om):
        phi = np.einsum("Ia,iab->Iib", phi, inst.tensors[k]).reshape(-1, chi)
    phi = phi @ inst.b_right                                       # [2^Omega]
    phi = phi.reshape([2] * Om)
    for s in _all_spins(6):
        # C_{s,i} = prod_j delta(s_j, i_w) for all w in R_j
        idx = tuple(int(s[p[w]]) for w in range(Om))
        assert _psi(o, s) == pytest.approx(phi[idx], rel=1e-11, abs=1e-300)
    # and C annihilates every replica configuration that breaks a constraint:
    # sum_s psi_s^2 equals the sum of phi^2 over constraint-respecting i only.
    tot = sum(_psi(o, s) ** 2 for s in _all_spins(6))
    assert tot < float(np.sum(phi ** 2))


def test_swap_spin_slices_maps_psi_to_complement():
    inst = _inst(np.tile(np.arange(6), 2), chi=4, seed=5)
    sw = _inst(inst.path, chi=4, seed=5, tensors=inst.tensors[:, ::-1].copy())
    sw.b_left, sw.b_right = inst.b_left, inst.b_right
    o, o2 = orc.Oracle(inst), orc.Oracle(sw)
    for s in _all_spins(6):
        assert o.amplitude(s) == o2.amplitude(1 - s)


def test_gauge_invariance():
    rng = np.random.default_rng(6)
    path = np.tile(np.arange(7), 2)
    L, chi = path.shape[0], 5
    inst = _inst(path, chi=chi, seed=7)
    G = [np.eye(chi)] + [np.linalg.qr(rng.standard_normal((chi, chi)))[0] for _ in range(L - 1)] + [np.eye(chi)]
    # A_k -> G_k^{-1} A_k G_{k+1}; boundary gauges are the identity
    t = np.stack([np.stack([G[k].T @ inst.tensors[k, s] @ G[k + 1] for s in (0, 1)]) for k in range(L)])
    g = _inst(path, chi=chi, seed=7, tensors=t)
    g.b_left, g.b_right = inst.b_left, inst.b_right
    o, og = orc.Oracle(inst), orc.Oracle(g)
    for _ in range(30):
        s = rng.integers(0, 2, 7).astype(np.uint8)
        assert _psi(og, s) == pytest.approx(_psi(o, s), rel=1e-12)


def test_power_of_two_rescale_is_exact():
    rng = np.random.default_rng(8)
    inst = _inst(np.tile(np.arange(6), 3), chi=4, seed=9)
    c = rng.integers(-40, 40, inst.path.shape[0])
    sc = _inst(inst.path, chi=4, seed=9, tensors=inst.tensors * np.ldexp(1.0, c)[:, None, None, None])
    sc.b_left, sc.b_right = inst.b_left, inst.b_right
    o, o2 = orc.Oracle(inst), orc.Oracle(sc)
    for _ in range(20):
        s = rng.integers(0, 2, 6).astype(np.uint8)
        m1, e1 = o.amplitude(s)
        m2, e2 = o2.amplitude(s)
        assert m1 == m2 and e2 - e1 == int(c.sum())


def test_flip_amplitude_equals_amplitude_of_flipped_state():
    rng = np.random.default_rng(10)
    order = inputs.snake_order(3, 4)
    inst = _inst(inputs.periodic_path(order, 3), chi=5, seed=11)
    o = orc.Oracle(inst)
    for _ in range(10):
        s = rng.integers(0, 2, 12).astype(np.uint8)
        for i in range(12):
            t = s.copy()
            t[i] ^= 1
            mf, ef = o.flip_amplitude(s, i)
            assert math.ldexp(mf, ef) == pytest.approx(_dense_product(inst, t), rel=1e-11)


def test_long_train_no_overflow():
    """L = 600 sites of entries ~ 1e3 would overflow a plain product (1e1800)."""
    inst = _inst(np.tile(np.arange(10), 60), chi=4, seed=12)
    inst.tensors *= 1e3
    o = orc.Oracle(inst)
    s = np.zeros(10, np.uint8)
    m, e = o.amplitude(s)
    assert 1.0 <= abs(m) < 2.0 and e > 1024


# --------------------------------------------------------------------------- energy

def _dense_tfim(n, bonds, J, h):
    """H = J sum Z_i Z_j - h sum X_i, basis index with spin 0 most significant,
    s = 0 <-> Z = +1."""
    I = np.eye(2)
    Z = np.diag([1.0, -1.0])
    X = np.array([[0.0, 1.0], [1.0, 0.0]])

    def op(site_ops):
        m = np.array([[1.0]])
        for i in range(n):
            m = np.kron(m, site_ops.get(i, I))
        return m
    H = np.zeros((1 << n, 1 << n))
    for i, j in bonds:
        H += J * op({int(i): Z, int(j): Z})
    for i in range(n):
        H -= h * op({i: X})
    return H


def test_local_energy_matches_dense_hamiltonian():
    lx, ly, R, chi = 3, 3, 2, 4
    inst = inputs.make_instance(lx, ly, R, chi, 3.0, seed=13, mixing=False)
    inst.J = 0.7
    o = orc.Oracle(inst)
    H = _dense_tfim(9, inst.bonds, inst.J, inst.h)
    psi = o.all_amplitudes()
    hpsi = H @ psi
    spins = _all_spins(9)
    eloc, ratios = o.local_energies(spins, with_ratios=True)
    np.testing.assert_allclose(eloc, hpsi / psi, rtol=1e-10, atol=1e-9)
    # ratios are psi(s^(i))/psi(s) with spin 0 the most significant bit
    for k in (0, 77, 300, 511):
        for i in range(9):
            assert ratios[k, i] == pytest.approx(psi[k ^ (1 << (8 - i))] / psi[k], rel=1e-11)
    e_exact = float(psi @ hpsi / (psi @ psi))
    assert o.exact_energy() == pytest.approx(e_exact, rel=1e-12)


def test_R1_transfer_matrix_energy_matches_enumeration():
    """R = 1: the RTT is an MPS (Sec. 2.1); its energy by transfer matrices."""
    inst = inputs.make_instance(4, 3, 1, 5, 2.5, seed=14, mixing=True)
    o = orc.Oracle(inst)
    assert o.exact_energy() == pytest.approx(orc.mps_energy(inst), rel=1e-10)


def _chi1_instance(R, lx, ly, seed):
    inst = inputs.make_instance(lx, ly, R, 1, 3.0, seed=seed, mixing=False)
    rng = np.random.default_rng(seed)
    inst.b_left = np.array([rng.uniform(0.5, 2)])
    inst.b_right = np.array([rng.uniform(0.5, 2)])
    return inst


def test_chi1_product_state_closed_form():
    inst = _chi1_instance(3, 3, 3, 15)
    o = orc.Oracle(inst)
    a = inst.tensors[:, :, 0, 0]                       # [L][2]
    c = np.ones((9, 2))
    for k, i in enumerate(inst.path):
        c[i] *= a[k]
    zi = (c[:, 0] ** 2 - c[:, 1] ** 2) / (c[:, 0] ** 2 + c[:, 1] ** 2)
    xi = 2 * c[:, 0] * c[:, 1] / (c[:, 0] ** 2 + c[:, 1] ** 2)
    e = inst.J * sum(zi[i] * zi[j] for i, j in inst.bonds) - inst.h * xi.sum()
    assert o.exact_energy() == pytest.approx(e, rel=1e-12)
    spins = _all_spins(9)[::7]
    eloc = o.local_energies(spins)
    for s, el in zip(spins, eloc):
        zz = sum((1 - 2 * int(s[i])) * (1 - 2 * int(s[j])) for i, j in inst.bonds)
        ref = inst.J * zz - inst.h * sum(c[i, 1 - s[i]] / c[i, s[i]] for i in range(9))
        assert el == pytest.approx(ref, rel=1e-12)


def test_equal_slices_all_ratios_one_and_all_flips_accepted():
    inst = inputs.make_instance(3, 3, 2, 4, 3.0, seed=16, mixing=True)
    inst.tensors[:, 1] = inst.tensors[:, 0]
    o = orc.Oracle(inst)
    spins = inputs.initial_spins(16, 8, 9)
    eloc, ratios = o.local_energies(spins, with_ratios=True)
    np.testing.assert_allclose(ratios, 1.0, rtol=1e-12)
    for s, el in zip(spins, eloc):
        zz = sum((1 - 2 * int(s[i])) * (1 - 2 * int(s[j])) for i, j in inst.bonds)
        assert el == pytest.approx(zz - 3.0 * 9, rel=1e-12)
    sp = spins.copy()
    mant, ex = o.init_chains(sp)
    _, acc = o.mcmc(5, sp, mant, ex, 0, 3)
    assert np.all(acc == 27)
    assert np.array_equal(sp, 1 - spins)      # three sweeps: every spin flipped thrice


# --------------------------------------------------------------------------- sampling

def test_mcmc_energy_matches_exact_enumeration():
    inst = inputs.workload("tiny_fp64")
    o = orc.Oracle(inst)
    B, T, burn = 64, 600, 100
    spins = inputs.initial_spins(1, B, inst.n_spins)
    mant, ex = o.init_chains(spins)
    o.mcmc(22719, spins, mant, ex, 0, burn, record=False, threads=8)
    trace, acc = o.mcmc(22719, spins, mant, ex, burn, T, threads=8)
    st = orc.observables(trace, inst.n_spins, acc, T * inst.n_spins)
    e = o.exact_energy()
    assert abs(st["mean"] - e) < 3.5 * st["se"], (st, e)
    assert 0.0 < st["accept_rate"] < 1.0


def test_mcmc_histogram_chi2_against_psi_squared():
    scipy_stats = pytest.importorskip("scipy.stats")
    inst = inputs.make_instance(3, 3, 2, 3, 3.0, seed=17, mixing=False)
    o = orc.Oracle(inst)
    psi = o.all_amplitudes()
    p = psi ** 2 / np.sum(psi ** 2)
    B = 12000
    spins = inputs.initial_spins(17, B, 9)
    mant, ex = o.init_chains(spins)
    o.mcmc(99, spins, mant, ex, 0, 25, record=False, threads=8)
    idx = np.zeros(B, dtype=np.int64)
    for i in range(9):
        idx = idx * 2 + spins[:, i]
    obs = np.bincount(idx, minlength=512).astype(float)
    exp = p * B
    order = np.argsort(exp)
    o_m, e_m, acc_o, acc_e = [], [], 0.0, 0.0
    for k in order:                       # merge smallest bins until expected >= 5
        acc_o += obs[k]
        acc_e += exp[k]
        if acc_e >= 5:
            o_m.append(acc_o)
            e_m.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0:
        o_m[-1] += acc_o
        e_m[-1] += acc_e
    chi2, pval = scipy_stats.chisquare(o_m, e_m)
    assert pval > 1e-3, (chi2, pval, len(o_m))


def test_chain_sharding_is_bit_identical():
    """Chain c's random stream depends on its global index only."""
    inst = inputs.make_instance(3, 3, 2, 4, 3.0, seed=18, mixing=True)
    o = orc.Oracle(inst)
    spins = inputs.initial_spins(18, 10, 9)
    a = spins.copy()
    ma, ea = o.init_chains(a)
    ta, _ = o.mcmc(7, a, ma, ea, 0, 5)
    b1, b2 = spins[:4].copy(), spins[4:].copy()
    m1, e1 = o.init_chains(b1)
    m2, e2 = o.init_chains(b2)
    t1, _ = o.mcmc(7, b1, m1, e1, 0, 5, chain0=0)
    t2, _ = o.mcmc(7, b2, m2, e2, 0, 5, chain0=4)
    assert np.array_equal(a, np.concatenate([b1, b2]))
    assert np.array_equal(ta, np.concatenate([t1, t2], axis=1))


def test_resume_is_bit_identical():
    inst = inputs.make_instance(3, 3, 2, 4, 3.0, seed=19, mixing=True)
    o = orc.Oracle(inst)
    s0 = inputs.initial_spins(19, 6, 9)
    a = s0.copy()
    ma, ea = o.init_chains(a)
    ta, acc_a = o.mcmc(3, a, ma, ea, 10, 6)
    b = s0.copy()
    mb, eb = o.init_chains(b)
    t1, acc1 = o.mcmc(3, b, mb, eb, 10, 2)
    t2, acc2 = o.mcmc(3, b, mb, eb, 12, 4)
    assert np.array_equal(a, b) and np.array_equal(ma, mb) and np.array_equal(ea, eb)
    assert np.array_equal(ta, np.concatenate([t1, t2]))
    assert np.array_equal(acc_a, acc1 + acc2)


# --------------------------------------------------------------------------- statistics

def test_tau_int_of_ar1_process():
    rng = np.random.default_rng(20)
    rho, T, B = 0.8, 20000, 32
    x = np.empty((T, B))
    x[0] = rng.standard_normal(B) / math.sqrt(1 - rho ** 2)
    eps = rng.standard_normal((T, B))
    for t in range(1, T):
        x[t] = rho * x[t - 1] + eps[t]
    tau, _ = orc.tau_int(x)
    assert tau == pytest.approx((1 + rho) / (2 * (1 - rho)), rel=0.08)


def test_observables_iid_and_vscore():
    rng = np.random.default_rng(21)
    x = 5.0 + 2.0 * rng.standard_normal((4000, 16))
    st = orc.observables(x, n_spins=10)
    assert st["tau_int"] == pytest.approx(0.5, abs=0.05)
    assert st["se"] == pytest.approx(2.0 / math.sqrt(x.size), rel=0.1)
    assert st["se_chain"] == pytest.approx(2.0 / math.sqrt(x.size), rel=0.5)
    assert st["v_score"] == pytest.approx(10 * st["var"] / st["mean"] ** 2, rel=1e-12)
    assert st["var"] == pytest.approx(4.0, rel=0.05)


# --------------------------------------------------------------------------- conditioning
# orc_amplitude_cond sets every floating-point tolerance of the FP32 and
# split-precision parity tests, so it is pinned by values worked out by hand
# from its definition: per site kappa_k = || |v| |A_k| ||_2 / || v A_k ||_2
# (v the incoming row after the exact power-of-two renormalisation), and
# kappa_fin = sum_b |v_b b_R[b]| / |sum_b v_b b_R[b]|.

def _cond(inst, s):
    return orc.Oracle(inst).amplitude_cond(np.asarray([s], dtype=np.uint8))[0]


def _one_site(A0, A1, bl, br):
    t = np.zeros((1, 2, 2, 2))
    t[0, 0], t[0, 1] = A0, A1
    return inputs.RTTInstance(n_spins=1, path=np.zeros(1, np.int32), tensors=t,
                              b_left=np.asarray(bl, float), b_right=np.asarray(br, float),
                              bonds=np.zeros((0, 2), np.int32), J=1.0, h=1.0)


def test_cond_positive_chi1_is_one_everywhere():
    """chi = 1 with positive entries: no cancellation anywhere, every kappa is
    exactly 1 (sum over L sites = L)."""
    L = 7
    rng = np.random.default_rng(3)
    t = rng.uniform(0.5, 2.0, size=(L, 2, 1, 1))
    inst = inputs.RTTInstance(n_spins=L, path=np.arange(L, dtype=np.int32), tensors=t,
                              b_left=np.ones(1), b_right=np.ones(1),
                              bonds=np.zeros((0, 2), np.int32), J=1.0, h=1.0)
    for s in ([0] * L, [1, 0, 1, 1, 0, 0, 1]):
        sk, mk, kf = _cond(inst, s)
        assert (sk, mk, kf) == (float(L), 1.0, 1.0)


def test_cond_two_by_two_by_hand():
    """One site, chi = 2, b_L = (1, 1), b_R = (1, -1).
    s = 0, A = [[1, -1], [2, 3]]: v A = (3, 2), |v||A| = (3, 4), so kappa =
    sqrt(25/13); the row renormalised by 2^-1 is (1.5, 1): kappa_fin =
    (1.5 + 1) / |1.5 - 1| = 5.
    s = 1, A = [[2, 0], [0, -1]]: v A = (2, -1) = |v||A| up to sign, kappa = 1;
    the row (1, -0.5) gives kappa_fin = 1.5 / 1.5 = 1."""
    inst = _one_site([[1.0, -1.0], [2.0, 3.0]], [[2.0, 0.0], [0.0, -1.0]], [1, 1], [1, -1])
    sk, mk, kf = _cond(inst, [0])
    assert sk == pytest.approx(math.sqrt(25.0 / 13.0), rel=1e-15)
    assert mk == sk and kf == 5.0
    assert tuple(_cond(inst, [1])) == (1.0, 1.0, 1.0)


def test_cond_closing_cancellation():
    """b_R = (1, -1.5 (1 - 2^-20)) against the row (1.5, 1): the closing sum is
    1.5 2^-20 and the absolute sum 3 - 1.5 2^-20, so kappa_fin = 2^21 - 1
    exactly."""
    eps = 2.0 ** -20
    inst = _one_site([[1.0, -1.0], [2.0, 3.0]], np.eye(2), [1, 1], [1.0, -1.5 * (1.0 - eps)])
    _, _, kf = _cond(inst, [0])
    assert kf == 2.0 ** 21 - 1.0


def test_cond_invariances_and_lower_bound():
    """kappa_k >= 1 and kappa_fin >= 1 (triangle inequality); scaling a site
    tensor by a power of two or negating it (both slices) leaves every kappa
    unchanged."""
    inst = inputs.make_instance(3, 3, 2, 6, 3.0, seed=21, mixing=True)
    spins = inputs.initial_spins(5, 6, 9)
    o = orc.Oracle(inst)
    base = o.amplitude_cond(spins)
    assert np.all(base[:, 1] >= 1.0) and np.all(base[:, 2] >= 1.0)
    assert np.all(base[:, 0] >= inst.path.shape[0])
    t = inst.tensors.copy()
    t[4] *= 8.0
    t[7] *= -1.0
    other = inputs.RTTInstance(n_spins=9, path=inst.path, tensors=t, b_left=inst.b_left,
                               b_right=inst.b_right, bonds=inst.bonds, J=inst.J, h=inst.h)
    np.testing.assert_allclose(orc.Oracle(other).amplitude_cond(spins), base, rtol=1e-13)


def test_replayed_sweep_reproduces_the_oracle_chain():
    """The teacher-forced replay of one sweep (the decisions read from the
    configuration after it) of the oracle's own chains finds every recorded
    decision equal to the rule u < r^2 and the uniforms of the Metropolis
    stream; a planted wrong decision is reported at its proposal."""
    inst = inputs.workload("tiny_fp64")
    o = orc.Oracle(inst)
    s0 = inputs.initial_spins(77, 48, inst.n_spins)
    s1 = s0.copy()
    m, e = o.init_chains(s1)
    o.mcmc(5, s1, m, e, 3, 1, record=False, chain0=10)
    r2, u, taken, rule, states = o.replay_sweep(5, s0, s1, 3, chain0=10, threads=4)
    assert np.array_equal(taken, rule)
    assert np.array_equal(states[:, 0], s0)
    assert u[2, 4] == orc.mcmc_uniform(5, 12, 3, 4)
    assert np.array_equal(taken, s1[:, inst.path[:inst.n_spins]] != s0[:, inst.path[:inst.n_spins]])
    bad = s1.copy()
    bad[7, inst.path[5]] ^= 1                     # proposal 5 of chain 7 decided the other way
    _, _, tk, ru, _ = o.replay_sweep(5, s0, bad, 3, chain0=10)
    first = np.argwhere(tk != ru)
    assert first[0].tolist() == [7, 5]
