"""Dual Monte Carlo of Sec. 3.3 in plain FP64 -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path (the CUDA library and
its Python binding) never calls it.

What it computes, for M RTTs psi^1..psi^M on one lattice and Hamiltonian:
  * ``direct_sum``: the linear combination sum_m c_m psi^m as one RTT.  A sum of
    tensor trains is a tensor train (Sec. 3.2, where psi' is turned back into
    an RTT by summing TTs): block-diagonal site tensors, the right boundary
    vectors stacked, the left ones stacked with the coefficients applied.
  * ``mixed_local_energies``: per configuration the mixed local energy
    E^{ab}(s) = sum_sbar H_{s,sbar} psi^b_sbar / psi^a_s and the overlap ratio
    r^{ab}(s) = psi^b_s / psi^a_s (C oracle, ``orc_mixed_local_energy``).
  * ``exact_tilde_matrices``: H~_ab = <E^{ab}>_{P^a} and S~_ab = <r^{ab}>_{P^a}
    with P^a = |psi^a|^2 / Z_a, by enumerating all 2^N configurations.
  * ``solve``: the generalized eigenproblem H~ c = lambda S~ c (Eq. gen_eig2)
    by a library eigen-solver; eigenvalues by increasing real part; the
    eigenvector of the lowest one scaled to |c^T S~ c| = 1 with its
    largest-magnitude entry positive.
  * ``gram_schmidt``: the matrix T of the stochastic Gram-Schmidt states
    psi'^m = psi^m - sum_{a<m} <psi^m / psi^a>_{P^a} psi^a (Eq. Gram-Schmid),
    i.e. T[m][a] = -S~_am below the unit diagonal (optionally against psi^1
    only, which the paper finds often sufficient); psi' = T psi.

Parity status: pinned in ``tests/test_oracle_dual.py`` against a dense TFIM
matrix and exact amplitude vectors (H_ab = psi^a . H . psi^b, S_ab =
psi^a . psi^b, Z_a H~_ab = H_ab), the identities S~_aa = 1 and H~_aa = <H>_a,
the projected symmetric eigenproblem, the variational bound, eigenvalue
invariance under the Gram-Schmidt change of basis, and direct-sum amplitudes
against the linear combination of amplitudes.
"""
from __future__ import annotations

import dataclasses
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from oracle.oracle import Oracle, _ptr


def _same_lattice(a, b):
    return (a.n_spins == b.n_spins and np.array_equal(a.path, b.path) and
            np.array_equal(np.asarray(a.bonds).reshape(-1, 2), np.asarray(b.bonds).reshape(-1, 2))
            and a.J == b.J and a.h == b.h)


def direct_sum(instances, coef):
    """One RTT whose amplitude is sum_m coef[m] psi^m (all on the same path)."""
    assert len(instances) == len(coef) >= 1
    first = instances[0]
    for other in instances[1:]:
        assert _same_lattice(first, other), "direct sum needs one path, bond list, J and h"
    L = first.path.shape[0]
    chis = [int(x.tensors.shape[2]) for x in instances]
    chi = sum(chis)
    t = np.zeros((L, 2, chi, chi))
    bl = np.zeros(chi)
    br = np.zeros(chi)
    off = 0
    for inst, c, x in zip(instances, coef, chis):
        t[:, :, off:off + x, off:off + x] = inst.tensors
        bl[off:off + x] = float(c) * np.asarray(inst.b_left)
        br[off:off + x] = np.asarray(inst.b_right)
        off += x
    return dataclasses.replace(first, tensors=t, b_left=bl, b_right=br,
                               name="sum(" + ",".join(i.name for i in instances) + ")")


def mixed_local_energies(oa: Oracle, ob: Oracle, spins, threads: int = 1):
    """(E^{ab}(s), r^{ab}(s)) for each row s of spins [B][N]."""
    spins = np.ascontiguousarray(spins, dtype=np.uint8)
    B = spins.shape[0]
    e = np.empty(B)
    r = np.empty(B)
    if threads <= 1 or B < 2 * threads:
        oa.lib.orc_mixed_local_energies(oa._p, ob._p, _ptr(spins), B, _ptr(e), _ptr(r))
        return e, r
    bounds = np.linspace(0, B, threads + 1).astype(np.int64)

    def run(t):
        a, b = bounds[t], bounds[t + 1]
        if b > a:
            oa.lib.orc_mixed_local_energies(oa._p, ob._p, _ptr(spins[a:b]), b - a,
                                            _ptr(e[a:b]), _ptr(r[a:b]))
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, range(threads)))
    return e, r


def all_configurations(n):
    """All 2^n configurations; row idx has s_i = bit (n-1-i) of idx."""
    idx = np.arange(1 << n, dtype=np.int64)
    return ((idx[:, None] >> (n - 1 - np.arange(n))[None, :]) & 1).astype(np.uint8)


def exact_tilde_matrices(instances, threads: int = 1):
    """(H~, S~) [M][M] by enumeration: H~_ab = sum_s P^a(s) E^{ab}(s)."""
    oracles = [Oracle(i) for i in instances]
    M = len(oracles)
    n = instances[0].n_spins
    spins = all_configurations(n)
    Ht = np.empty((M, M))
    St = np.empty((M, M))
    for a, oa in enumerate(oracles):
        psi = oa.all_amplitudes()
        p = psi * psi
        p = p / p.sum()
        for b, ob in enumerate(oracles):
            e, r = mixed_local_energies(oa, ob, spins, threads)
            keep = p > 0
            Ht[a, b] = float(np.sum(p[keep] * e[keep]))
            St[a, b] = float(np.sum(p[keep] * r[keep]))
    return Ht, St


def solve(Ht, St):
    """Eigenvalues of H~ c = lambda S~ c by increasing real part, and the
    eigenvector of the first (real part) scaled as described above."""
    import scipy.linalg
    w, v = scipy.linalg.eig(np.asarray(Ht, dtype=np.float64), np.asarray(St, dtype=np.float64))
    order = np.lexsort((w.imag, w.real))
    w = w[order]
    c = np.real(v[:, order[0]]).astype(np.float64)
    q = float(c @ np.asarray(St) @ c)
    if q != 0.0 and np.isfinite(q):
        c = c / np.sqrt(abs(q))
    k = int(np.argmax(np.abs(c)))
    if c[k] < 0:
        c = -c
    return w, c


def gram_schmidt(St, first_only: bool = False):
    """T with psi' = T psi for the stochastic Gram-Schmidt states."""
    St = np.asarray(St, dtype=np.float64)
    M = St.shape[0]
    T = np.eye(M)
    for m in range(1, M):
        for a in range(1 if first_only else m):
            T[m, a] = -St[a, m]
    return T
