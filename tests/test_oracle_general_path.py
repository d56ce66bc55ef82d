"""The oracle on general paths (the replicas visit the spins in different
orders, Sec. 2.2.1 path sums; orderings of Sec. 4): pinned against brute
force and a dense TFIM matrix."""

import numpy as np
import pytest

from paper_2604_22718_gb300 import inputs
from oracle import oracle as orc
from oracle import dual


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


@pytest.mark.parametrize("lx,ly", [(3, 3), (4, 3), (6, 6)])
def test_orderings_are_permutations_and_snakes(lx, ly):
    for name in ("H", "V", "D", "Dp"):
        o = inputs.ordering(name, lx, ly)
        assert sorted(o.tolist()) == list(range(lx * ly))
    # row and column snakes move to a lattice neighbour at every step
    for name in ("H", "V"):
        o = inputs.ordering(name, lx, ly)
        for a, b in zip(o[:-1], o[1:]):
            ax, ay, bx, by = a % lx, a // lx, b % lx, b // lx
            assert abs(ax - bx) + abs(ay - by) == 1
    # the diagonal snakes keep x + y (x - y) non-decreasing along the path
    d = [i % lx + i // lx for i in inputs.ordering("D", lx, ly)]
    dp = [i % lx - i // lx for i in inputs.ordering("Dp", lx, ly)]
    assert d == sorted(d) and dp == sorted(dp)


def test_path_sum_concatenates():
    p = inputs.path_sum([inputs.ordering("V", 3, 3), inputs.ordering("H", 3, 3)])
    assert p.tolist() == inputs.ordering("V", 3, 3).tolist() + inputs.ordering("H", 3, 3).tolist()


def test_general_path_amplitude_flip_and_energy_by_brute_force():
    inst = inputs.make_path_instance(3, 3, ("V", "H", "D", "Dp"), 3, 3.0, seed=21)
    o = orc.Oracle(inst)
    spins = dual.all_configurations(9)
    psi = o.all_amplitudes()
    # amplitude = dense product along the path
    for s in spins[::37]:
        mats = [inst.tensors[k, s[inst.path[k]]] for k in range(inst.path.shape[0])]
        want = float(inst.b_left @ np.linalg.multi_dot(mats + [inst.b_right]))
        m, e = o.amplitude(s)
        assert np.ldexp(m, e) == pytest.approx(want, rel=1e-11)
    # flip amplitude = amplitude of the flipped configuration
    for s in spins[::53]:
        for i in range(9):
            t = s.copy()
            t[i] ^= 1
            mf, ef = o.flip_amplitude(s, i)
            mt, et = o.amplitude(t)
            assert np.ldexp(mf, ef) == pytest.approx(np.ldexp(mt, et), rel=1e-11)
    # E_loc against the dense Hamiltonian
    H = _dense_tfim(9, inst.bonds, inst.J, inst.h)
    e = o.local_energies(spins)
    np.testing.assert_allclose(e, (H @ psi) / psi, rtol=1e-10, atol=1e-10)
