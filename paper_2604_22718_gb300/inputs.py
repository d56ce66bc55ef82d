"""Seeded synthetic inputs for the RTT sampler.

This module only *generates data*: lattice orderings, bond lists, RTT tensors
and initial spin configurations.  It contains none of the method's arithmetic
(no amplitude, ratio, energy or acceptance computation), so both the CUDA path
and the FP64 oracle may consume what it produces.

Workloads (2D transverse-field Ising model on open Lx x Ly lattices, Sec. 4,
Eq. ising-model; RTT path = a lattice ordering repeated R times, the path sum
of Sec. 2.2.1):

* ``tiny_fp64``   3x3, R=2, chi=8,   h=3.0,   iid N(0,1)/sqrt(chi) tensors
* ``plain_6x6``   6x6, R=2, chi=64,  h=3.0,   Gaussian/sqrt(chi) x Haar Q_k
* ``prec_10x10``  10x10, R=3, chi=128, h=3.04, same generator
* ``learned_16x16`` 16x16, R=2, chi=128, h=3.044, same generator
* ``batched64``   64 instances, Lx in {4,6,8,12}, R in {2,3,4},
                  chi in {32,64,128,256}, h ~ U[2.5,3.5]
* ``dual_6x6``    3 states of the plain_6x6 kind (dual Monte Carlo)
* ``vhdd_6x6``    6x6, path sigma^V + sigma^H + sigma^D + sigma^D' (R = 4, L = 144), chi = 64
* ``replica_*``   replica-space optimization (Sec. 3.1, Sec. 4): 6x6, 10x10, 20x20 on
                  sigma^V + sigma^H + sigma^D + sigma^D', chi = 2, tau = 0.1, h = 3, H-bar_HV

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "RTTInstance", "snake_order", "column_snake", "diagonal_snake", "ordering", "path_sum",
    "make_path_instance", "open_bonds", "periodic_path",
    "gaussian_tensors", "mixed_tensors", "make_instance", "initial_spins",
    "WORKLOADS", "workload", "workload_states", "batched_instances", "made_init_weights", "ferro_chain_instance",
    "BOND_STEPS", "direction_bonds", "replica_terms", "hbar_terms", "terms_arrays", "replica_start",
    "replica_ones", "REPLICA_WORKLOADS",
]


@dataclasses.dataclass
class RTTInstance:
    """Plain container for one RTT state and its TFIM Hamiltonian."""
    n_spins: int
    path: np.ndarray        # int32 [L], path[k] = spin tied to train site k
    tensors: np.ndarray     # float64 [L][2][chi][chi], A_k[s][a][b]
    b_left: np.ndarray      # float64 [chi]
    b_right: np.ndarray     # float64 [chi]
    bonds: np.ndarray       # int32 [n_bonds][2]
    J: float
    h: float
    name: str = ""
    lx: int = 0
    ly: int = 0
    R: int = 0

    @property
    def length(self) -> int:
        return int(self.path.shape[0])

    @property
    def chi(self) -> int:
        return int(self.tensors.shape[2])


def snake_order(lx: int, ly: int) -> np.ndarray:
    """Boustrophedon ordering of an lx x ly lattice, site index i = y*lx + x.

    Row y is walked left-to-right for even y and right-to-left for odd y."""
    out = []
    for y in range(ly):
        xs = range(lx) if y % 2 == 0 else range(lx - 1, -1, -1)
        out.extend(y * lx + x for x in xs)
    return np.asarray(out, dtype=np.int32)


def column_snake(lx: int, ly: int) -> np.ndarray:
    """Column by column (sigma^V): column x walked with increasing y for even x,
    decreasing y for odd x; site index i = y*lx + x."""
    out = []
    for x in range(lx):
        ys = range(ly) if x % 2 == 0 else range(ly - 1, -1, -1)
        out.extend(y * lx + x for y in ys)
    return np.asarray(out, dtype=np.int32)


def diagonal_snake(lx: int, ly: int, anti: bool = False) -> np.ndarray:
    """Diagonal by diagonal (sigma^D: x + y constant; sigma^D' with anti=True:
    x - y constant), diagonal number d walked with increasing x for even d,
    decreasing x for odd d."""
    out = []
    n_diag = lx + ly - 1
    for d in range(n_diag):
        cells = []
        for x in range(lx):
            y = (d - x) if not anti else (x - d + ly - 1)
            if 0 <= y < ly:
                cells.append(y * lx + x)
        out.extend(cells if d % 2 == 0 else cells[::-1])
    return np.asarray(out, dtype=np.int32)


def ordering(name: str, lx: int, ly: int) -> np.ndarray:
    """One of the orderings of Sec. 4: 'H' (rows), 'V' (columns), 'D', 'Dp'."""
    return {"H": lambda: snake_order(lx, ly), "V": lambda: column_snake(lx, ly),
            "D": lambda: diagonal_snake(lx, ly), "Dp": lambda: diagonal_snake(lx, ly, anti=True)}[name]()


def path_sum(orders) -> np.ndarray:
    """sigma^1 + sigma^2 + ...: the orderings one after the other (Sec. 2.2.1)."""
    return np.concatenate([np.asarray(o, dtype=np.int32) for o in orders])


def make_path_instance(lx: int, ly: int, names, chi: int, h: float, seed: int,
                       mixing: bool = True, J: float = 1.0, name: str = "") -> RTTInstance:
    """An RTT on the path sigma^{names[0]} + sigma^{names[1]} + ... (one replica
    per ordering), tensors as make_instance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    path = path_sum([ordering(n, lx, ly) for n in names])
    L = path.shape[0]
    t = mixed_tensors(rng, L, chi) if mixing else gaussian_tensors(rng, L, chi)
    ones = np.ones(chi, dtype=np.float64)
    return RTTInstance(n_spins=lx * ly, path=path, tensors=np.ascontiguousarray(t),
                       b_left=ones.copy(), b_right=ones.copy(), bonds=open_bonds(lx, ly),
                       J=float(J), h=float(h), name=name, lx=lx, ly=ly, R=len(names))


def open_bonds(lx: int, ly: int) -> np.ndarray:
    """Nearest-neighbour bonds of an open lx x ly square lattice."""
    b = []
    for y in range(ly):
        for x in range(lx):
            i = y * lx + x
            if x + 1 < lx:
                b.append((i, i + 1))
            if y + 1 < ly:
                b.append((i, i + lx))
    return np.asarray(b, dtype=np.int32).reshape(-1, 2)


def periodic_path(order: np.ndarray, R: int) -> np.ndarray:
    """The ordering repeated R times (path sum of R copies)."""
    return np.tile(np.asarray(order, dtype=np.int32), R)


def gaussian_tensors(rng: np.random.Generator, L: int, chi: int) -> np.ndarray:
    """A_k[s][a][b] i.i.d. N(0,1)/sqrt(chi)."""
    return rng.standard_normal((L, 2, chi, chi)) / np.sqrt(chi)


def _haar_orthogonal(rng: np.random.Generator, chi: int) -> np.ndarray:
    g = rng.standard_normal((chi, chi))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def mixed_tensors(rng: np.random.Generator, L: int, chi: int) -> np.ndarray:
    """A_k[s] = (G_k[s]/sqrt(chi)) Q_k with one Haar-random orthogonal Q_k per site."""
    g = rng.standard_normal((L, 2, chi, chi)) / np.sqrt(chi)
    out = np.empty_like(g)
    for k in range(L):
        q = _haar_orthogonal(rng, chi)
        out[k, 0] = g[k, 0] @ q
        out[k, 1] = g[k, 1] @ q
    return out


def make_instance(lx: int, ly: int, R: int, chi: int, h: float, seed: int,
                  mixing: bool = True, J: float = 1.0, name: str = "") -> RTTInstance:
    rng = np.random.Generator(np.random.PCG64(seed))
    order = snake_order(lx, ly)
    path = periodic_path(order, R)
    L = path.shape[0]
    t = mixed_tensors(rng, L, chi) if mixing else gaussian_tensors(rng, L, chi)
    ones = np.ones(chi, dtype=np.float64)
    return RTTInstance(n_spins=lx * ly, path=path, tensors=np.ascontiguousarray(t),
                       b_left=ones.copy(), b_right=ones.copy(),
                       bonds=open_bonds(lx, ly), J=float(J), h=float(h), name=name,
                       lx=lx, ly=ly, R=R)


def initial_spins(seed: int, n_chains: int, n_spins: int) -> np.ndarray:
    """uint8 [n_chains][n_spins], uniform random bits (seed stream separate from tensors)."""
    rng = np.random.Generator(np.random.PCG64([seed, 0x5350494e]))
    return rng.integers(0, 2, size=(n_chains, n_spins), dtype=np.uint8)


# name -> (lx, ly, R, chi, h, mixing, chains, sweeps, seed)
WORKLOADS = {
    "tiny_fp64":     dict(lx=3, ly=3, R=2, chi=8, h=3.0, mixing=False, chains=64, sweeps=1000, seed=22719),
    "plain_6x6":     dict(lx=6, ly=6, R=2, chi=64, h=3.0, mixing=True, chains=4096, sweeps=2000, seed=22720),
    "prec_10x10":    dict(lx=10, ly=10, R=3, chi=128, h=3.04, mixing=True, chains=16384, sweeps=1000, seed=22721),
    "learned_16x16": dict(lx=16, ly=16, R=2, chi=128, h=3.044, mixing=True, chains=8192, sweeps=128, seed=22723),
    # the same state and chains with local flips only (the plain sampler the
    # learned proposal is compared with)
    "plain_16x16":   dict(lx=16, ly=16, R=2, chi=128, h=3.044, mixing=True, chains=8192, sweeps=128, seed=22723),
    # the path sigma^V + sigma^H + sigma^D + sigma^D' of Sec. 4 (four replicas), FP32/FP64 sampler
    "vhdd_6x6":      dict(lx=6, ly=6, R=4, chi=64, h=3.0, mixing=True, chains=4096, sweeps=100, seed=22729,
                          orderings=("V", "H", "D", "Dp")),
    # dual Monte Carlo: M = 3 states of the plain_6x6 kind (seeds seed, seed+1, seed+2)
    "dual_6x6":      dict(lx=6, ly=6, R=2, chi=64, h=3.0, mixing=True, chains=4096, sweeps=100, seed=22726, states=3),
}


def workload(name: str, **override) -> RTTInstance:
    w = dict(WORKLOADS[name])
    w.update(override)
    if "orderings" in w:
        return make_path_instance(w["lx"], w["ly"], w["orderings"], w["chi"], w["h"], w["seed"],
                                  mixing=w["mixing"], name=name)
    return make_instance(w["lx"], w["ly"], w["R"], w["chi"], w["h"], w["seed"],
                         mixing=w["mixing"], name=name)


def workload_states(name: str) -> list:
    """The M states of a multi-state workload (seeds seed .. seed + M - 1)."""
    w = WORKLOADS[name]
    return [make_instance(w["lx"], w["ly"], w["R"], w["chi"], w["h"], w["seed"] + m,
                          mixing=w["mixing"], name=f"{name}[{m}]") for m in range(w["states"])]


def batched_instances(seed: int = 22722, n: int = 64, chi_choices=(32, 64, 128, 256),
                      sizes=(4, 6, 8, 12), reps=(2, 3, 4)) -> list:
    """64 independent instances with lattice, R, chi and h drawn from the seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for t in range(n):
        lx = int(rng.choice(sizes))
        R = int(rng.choice(reps))
        chi = int(rng.choice(chi_choices))
        h = float(rng.uniform(2.5, 3.5))
        out.append(make_instance(lx, lx, R, chi, h, seed * 1000 + t, mixing=True,
                                 name=f"batched[{t}]"))
    return out


def made_init_weights(seed: int, n_spins: int, hidden: int) -> np.ndarray:
    """Initial weights of the autoregressive proposal network, flat float64 in
    the order W1 [H,N], b1 [H], W2 [H,H], b2 [H], W3 [N,H], b3 [N]: weights
    U(-1, 1)/sqrt(fan_in), biases zero.  Unmasked (masking is the model's)."""
    rng = np.random.Generator(np.random.PCG64([seed, 0x4D414445]))
    N, H = int(n_spins), int(hidden)
    parts = [rng.uniform(-1, 1, (H, N)) / np.sqrt(N), np.zeros(H),
             rng.uniform(-1, 1, (H, H)) / np.sqrt(H), np.zeros(H),
             rng.uniform(-1, 1, (N, H)) / np.sqrt(H), np.zeros(N)]
    return np.concatenate([x.ravel() for x in parts])


def ferro_chain_instance(lx: int, ly: int, kappa: float, field: float = 0.0, h: float = 3.0,
                         R: int = 1) -> RTTInstance:
    """An RTT whose amplitude is exp(kappa sum_k z_k z_(k+1) + field sum_k z_k)
    along the snake ordering (a ferromagnetic chain; bond index = previous
    spin), chi = 2; with R > 1 the extra blocks carry identity slices.  Local
    single-spin moves mix it slowly for large kappa; the field makes the two
    polarised modes unequal."""
    order = snake_order(lx, ly)
    N = lx * ly
    path = periodic_path(order, R)
    L = path.shape[0]
    t = np.zeros((L, 2, 2, 2))
    for k in range(L):
        for s in (0, 1):
            z = 1 - 2 * s
            for a in (0, 1):
                if k >= N:
                    t[k, s, a, a] = 1.0
                    continue
                w = float(np.exp(field * z))
                if k > 0:
                    w *= float(np.exp(kappa * (1 - 2 * a) * z))
                t[k, s, a, s] = w
    ones = np.ones(2)
    return RTTInstance(n_spins=N, path=path, tensors=t, b_left=ones.copy(), b_right=ones.copy(),
                       bonds=open_bonds(lx, ly), J=1.0, h=float(h), name=f"ferro{lx}x{ly}",
                       lx=lx, ly=ly, R=R)


# ---------------------------------------------------------------- replica-space optimization
# Physical operators of Sec. 4 as lists of Pauli terms, each with the replica
# block its Z factors are sent to (the "-> C" choice of Sec. 4).  Only the
# operator's definition lives here; lifting it to the replica space is the
# method's and is done by the library (and, independently, by the oracle).

BOND_STEPS = {"H": (1, 0), "V": (0, 1), "D": (1, -1), "Dp": (1, 1)}


def direction_bonds(lx: int, ly: int, direction: str) -> np.ndarray:
    """Nearest-neighbour pairs (i, j), i = y*lx + x, along one direction.

    'H' and 'V' are the horizontal and vertical bonds; 'D' pairs neighbours on
    the diagonals x + y = const that sigma^D walks, 'Dp' those on x - y = const
    that sigma^D' walks, so that a term sent to its own ordering is local."""
    dx, dy = BOND_STEPS[direction]
    out = []
    for y in range(ly):
        for x in range(lx):
            x2, y2 = x + dx, y + dy
            if 0 <= x2 < lx and 0 <= y2 < ly:
                out.append((y * lx + x, y2 * lx + x2))
    return np.asarray(out, dtype=np.int32).reshape(-1, 2)


def replica_terms(lx: int, ly: int, orderings, zz, h: float, x_block: int = 0):
    """Terms of sum_(d, c, target) c O_{ZZ, d -> target} - h O_X.

    zz: list of (direction, coefficient, target ordering name); the ZZ terms of
    each entry are sent to the block of ``orderings`` with that name.  Returns
    a list of (coef, [(spin, 'Z'|'X'), ...], block), in the order: the zz
    entries as given (bonds by site index), then the transverse-field terms
    (site index order).  X factors go to every replica whatever the block."""
    orderings = list(orderings)
    terms = []
    for direction, coef, target in zz:
        blk = orderings.index(target)
        for i, j in direction_bonds(lx, ly, direction):
            terms.append((float(coef), [(int(i), "Z"), (int(j), "Z")], blk))
    if h != 0.0:
        for i in range(lx * ly):
            terms.append((-float(h), [(i, "X")], int(x_block)))
    return terms


def hbar_terms(kind: str, lx: int, ly: int, h: float, orderings=("V", "H", "D", "Dp"),
               J: float = 1.0, alpha: float = 0.08):
    """The replica Hamiltonians of Sec. 4 (Eq. H_HV and the two around it):
    'H' (all ZZ terms on the H ordering), 'HV' (horizontal bonds on H, vertical
    on V), 'HVDDp' ('HV' plus alpha times the diagonal bonds on D and D')."""
    zz = {"H": [("H", J, "H"), ("V", J, "H")],
          "HV": [("H", J, "H"), ("V", J, "V")],
          "HVDDp": [("H", J, "H"), ("V", J, "V"), ("D", alpha, "D"), ("Dp", alpha, "Dp")]}[kind]
    return replica_terms(lx, ly, orderings, zz, h)


def terms_arrays(terms):
    """Flatten a term list for the C ABI: coef [K] f64, block [K] i32,
    offsets [K+1] i32, spins [F] i32, ops [F] u8 ('X' = 1, 'Z' = 2)."""
    code = {"X": 1, "Z": 2, "Y": 3}
    coef = np.asarray([t[0] for t in terms], dtype=np.float64)
    block = np.asarray([t[2] for t in terms], dtype=np.int32)
    off = np.zeros(len(terms) + 1, dtype=np.int32)
    spins, ops = [], []
    for k, (_, factors, _) in enumerate(terms):
        for j, op in factors:
            spins.append(int(j))
            ops.append(code[op])
        off[k + 1] = len(spins)
    return (coef, block, off, np.asarray(spins, dtype=np.int32), np.asarray(ops, dtype=np.uint8))


def replica_start(seed, L: int, chi: int) -> np.ndarray:
    """A random starting TT, padded cores [L][2][chi][chi] (row = left bond):
    Gaussian entries / sqrt(2 chi) on ranks min(chi, 2^k, 2^(L-k)), zeros
    elsewhere (the first core has one row, the last one column)."""
    rng = np.random.Generator(np.random.PCG64([int(seed), 0x52455043]))
    r = [min(chi, 2 ** min(k, 62), 2 ** min(L - k, 62)) for k in range(L + 1)]
    out = np.zeros((L, 2, chi, chi))
    for k in range(L):
        out[k, :, :r[k], :r[k + 1]] = rng.standard_normal((2, r[k], r[k + 1])) / np.sqrt(2 * chi)
    return out


def replica_ones(L: int, chi: int) -> np.ndarray:
    """phi^(0)_i = 1 for every i (the paper's starting TT), padded cores."""
    out = np.zeros((L, 2, chi, chi))
    out[:, :, 0, 0] = 1.0
    return out


REPLICA_WORKLOADS = {
    # the paper's replica-space runs: chi = 2, tau = 0.1, h = 3, path sigma^V+H+D+D'
    "replica_6x6":   dict(lx=6, ly=6, orderings=("V", "H", "D", "Dp"), chi=2, tau=0.1, h=3.0,
                          kind="HV", steps=200),
    "replica_10x10": dict(lx=10, ly=10, orderings=("V", "H", "D", "Dp"), chi=2, tau=0.1, h=3.0,
                          kind="HV", steps=200),
    "replica_20x20": dict(lx=20, ly=20, orderings=("V", "H", "D", "Dp"), chi=2, tau=0.1, h=3.0,
                          kind="HV", steps=50),
}
