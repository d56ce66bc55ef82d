"""FP64 CPU oracle for the RTT Monte Carlo hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path (the CUDA library and
its Python binding) never calls it.

Parts:
  * ctypes front-end to ``rtt_oracle.c`` (amplitudes, flip amplitudes, local
    energies, Metropolis, exact enumeration, Philox4x64-10);
  * plain numpy statistics of a local-energy trace (mean, variance, Sokal
    automatic-window integrated autocorrelation time, effective sample size,
    binned and tau-based standard errors, V-score N var/E^2 of Sec. 4.3).

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (brute-force dense contraction, the
constraint formulation psi = C phi of Sec. 2.2.3, the worked 6-spin example of
Sec. 2.2.1, a dense TFIM matrix, MPS transfer matrices at R = 1, closed forms
at chi = 1, numpy's Philox, AR(1) processes).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rtt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, no implicit fma contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Rtt(ctypes.Structure):
    _fields_ = [("n_spins", ctypes.c_int32), ("length", ctypes.c_int32),
                ("chi", ctypes.c_int32), ("n_bonds", ctypes.c_int32),
                ("path", ctypes.c_void_p), ("tensors", ctypes.c_void_p),
                ("b_left", ctypes.c_void_p), ("b_right", ctypes.c_void_p),
                ("bonds", ctypes.c_void_p), ("J", ctypes.c_double), ("h", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            U64 = ctypes.c_uint64
            lib.orc_amplitude.argtypes = [P, P, P, P]
            lib.orc_flip_amplitude.argtypes = [P, P, ctypes.c_int, P, P]
            lib.orc_local_energy.argtypes = [P, P, P, P]
            lib.orc_local_energy.restype = ctypes.c_int
            lib.orc_philox4x64.argtypes = [P, P, P]
            lib.orc_mcmc_uniform.argtypes = [U64, U64, U64, U64]
            lib.orc_mcmc_uniform.restype = ctypes.c_double
            lib.orc_mcmc.argtypes = [P, U64, P, P, P, I64, I64, I64, ctypes.c_int32,
                                     ctypes.c_int32, P, P]
            lib.orc_mcmc.restype = ctypes.c_int
            lib.orc_all_amplitudes.argtypes = [P, P]
            lib.orc_exact_energy.argtypes = [P, P]
            lib.orc_exact_energy.restype = ctypes.c_double
            lib.orc_log_amplitudes.argtypes = [P, P, I64, P, P, P, P]
            lib.orc_local_energies.argtypes = [P, P, I64, P, P]
            lib.orc_local_energies.restype = ctypes.c_int
            lib.orc_flip_amplitudes.argtypes = [P, P, I64, P, P]
            lib.orc_amplitude_cond.argtypes = [P, P, P, P, P]
            lib.orc_mixed_local_energy.argtypes = [P, P, P, P, P]
            lib.orc_mixed_local_energy.restype = ctypes.c_int
            lib.orc_mixed_local_energies.argtypes = [P, P, P, I64, P, P]
            lib.orc_mixed_local_energies.restype = ctypes.c_int
            lib.orc_uniform_keyed.argtypes = [U64, U64, U64, U64, U64]
            lib.orc_uniform_keyed.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class Oracle:
    """Holds contiguous copies of one RTT instance for the C oracle."""

    def __init__(self, inst):
        self.inst = inst
        self.n = int(inst.n_spins)
        self.path = np.ascontiguousarray(inst.path, dtype=np.int32)
        self.tensors = np.ascontiguousarray(inst.tensors, dtype=np.float64)
        self.bl = np.ascontiguousarray(inst.b_left, dtype=np.float64)
        self.br = np.ascontiguousarray(inst.b_right, dtype=np.float64)
        self.bonds = np.ascontiguousarray(inst.bonds, dtype=np.int32).reshape(-1, 2)
        L, two, chi, chi2 = self.tensors.shape
        assert two == 2 and chi == chi2 and L == self.path.shape[0]
        self.chi = chi
        self.L = L
        self._s = _Rtt(self.n, L, chi, self.bonds.shape[0], self.path.ctypes.data,
                       self.tensors.ctypes.data, self.bl.ctypes.data, self.br.ctypes.data,
                       self.bonds.ctypes.data if self.bonds.size else None,
                       float(inst.J), float(inst.h))
        self.lib = _load()

    @property
    def _p(self):
        return ctypes.byref(self._s)

    # -- amplitudes ---------------------------------------------------------
    def amplitude(self, s):
        """(mant, exp): psi(s) = mant * 2**exp, |mant| in [1,2)."""
        s = np.ascontiguousarray(s, dtype=np.uint8)
        m = ctypes.c_double()
        e = ctypes.c_int64()
        self.lib.orc_amplitude(self._p, _ptr(s), ctypes.byref(m), ctypes.byref(e))
        return m.value, e.value

    def flip_amplitude(self, s, i):
        s = np.ascontiguousarray(s, dtype=np.uint8)
        m = ctypes.c_double()
        e = ctypes.c_int64()
        self.lib.orc_flip_amplitude(self._p, _ptr(s), int(i), ctypes.byref(m), ctypes.byref(e))
        return m.value, e.value

    def log_amplitudes(self, spins):
        spins = np.ascontiguousarray(spins, dtype=np.uint8)
        B = spins.shape[0]
        la = np.empty(B)
        sg = np.empty(B, dtype=np.int8)
        mant = np.empty(B)
        ex = np.empty(B, dtype=np.int64)
        self.lib.orc_log_amplitudes(self._p, _ptr(spins), B, _ptr(la), _ptr(sg), _ptr(mant), _ptr(ex))
        return la, sg, mant, ex

    def flip_amplitudes(self, spins):
        spins = np.ascontiguousarray(spins, dtype=np.uint8)
        B = spins.shape[0]
        mant = np.empty((B, self.n))
        ex = np.empty((B, self.n), dtype=np.int64)
        self.lib.orc_flip_amplitudes(self._p, _ptr(spins), B, _ptr(mant), _ptr(ex))
        return mant, ex

    def local_energies(self, spins, with_ratios=False, threads: int = 1):
        spins = np.ascontiguousarray(spins, dtype=np.uint8)
        B = spins.shape[0]
        e = np.empty(B)
        r = np.empty((B, self.n)) if with_ratios else None
        if threads <= 1 or B < 2 * threads:
            self.lib.orc_local_energies(self._p, _ptr(spins), B, _ptr(e), _ptr(r))
            return (e, r) if with_ratios else e
        bounds = np.linspace(0, B, threads + 1).astype(np.int64)

        def run(t):
            a, b = bounds[t], bounds[t + 1]
            if b <= a:
                return
            sp = spins[a:b]
            ee = e[a:b]
            rr = r[a:b] if r is not None else None
            self.lib.orc_local_energies(self._p, _ptr(sp), b - a, _ptr(ee), _ptr(rr))
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, range(threads)))
        return (e, r) if with_ratios else e

    def amplitude_cond(self, spins, threads: int = 0):
        """Per configuration: (sum_k kappa_k, max_k kappa_k, kappa_fin) of the
        left-to-right evaluation (see orc_amplitude_cond); configurations
        spread over `threads` host threads (0: all cores)."""
        spins = np.ascontiguousarray(spins, dtype=np.uint8)
        B = spins.shape[0]
        out = np.empty((B, 3))

        def run(c):
            a, b, k = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            self.lib.orc_amplitude_cond(self._p, _ptr(spins[c]), ctypes.byref(a),
                                        ctypes.byref(b), ctypes.byref(k))
            out[c] = (a.value, b.value, k.value)
        nt = min(threads or (os.cpu_count() or 1), B)
        if nt <= 1 or B * self.L * self.chi * self.chi < (1 << 22):
            for c in range(B):
                run(c)
        else:
            with ThreadPoolExecutor(nt) as ex:
                list(ex.map(run, range(B)))
        return out

    def all_amplitudes(self):
        assert self.n <= 22
        psi = np.empty(1 << self.n)
        self.lib.orc_all_amplitudes(self._p, _ptr(psi))
        return psi

    def exact_energy(self):
        assert self.n <= 22
        nrm = ctypes.c_double()
        e = self.lib.orc_exact_energy(self._p, ctypes.byref(nrm))
        return e

    # -- Metropolis -----------------------------------------------------------
    def init_chains(self, spins):
        _, _, mant, ex = self.log_amplitudes(spins)
        return mant, ex

    def mcmc(self, seed, spins, mant, ex, sweep0, n_sweeps, measure_every=1,
             chain0=0, threads: int = 1, record=True):
        """Runs the sampler in place on (spins, mant, ex).  Returns (trace, n_accept);
        trace[g] is E_loc of the configuration entering sweep g * measure_every."""
        assert spins.flags.c_contiguous and spins.dtype == np.uint8
        assert mant.flags.c_contiguous and ex.flags.c_contiguous
        B = spins.shape[0]
        n_meas = n_sweeps // measure_every if (record and measure_every > 0) else 0
        trace = np.empty((n_meas, B)) if n_meas > 0 else None
        acc = np.zeros(B, dtype=np.int64)
        if threads <= 1 or B < 2 * threads:
            parts = [(0, B)]
        else:
            b = np.linspace(0, B, threads + 1).astype(np.int64)
            parts = [(int(b[t]), int(b[t + 1])) for t in range(threads) if b[t + 1] > b[t]]

        def run(part):
            a, b = part
            n = b - a
            tr = np.empty((n_meas, n)) if n_meas > 0 else None
            sp = spins[a:b]
            mm = mant[a:b]
            ee = ex[a:b]
            aa = acc[a:b]
            self.lib.orc_mcmc(self._p, int(seed), _ptr(sp), _ptr(mm), _ptr(ee), n,
                              int(chain0 + a), int(sweep0), int(n_sweeps),
                              int(measure_every if n_meas > 0 else 0), _ptr(tr), _ptr(aa))
            if tr is not None:
                trace[:, a:b] = tr
        if len(parts) == 1:
            run(parts[0])
        else:
            with ThreadPoolExecutor(len(parts)) as exe:
                list(exe.map(run, parts))
        return trace, acc


    def replay_sweep(self, seed, s_before, s_after, sweep, chain0=0, threads: int = 1):
        """One systematic sweep (Sec. 3.3: proposal j flips spin path[j], accept
        iff u < (psi(s')/psi(s))^2) of every chain, taking the decisions that
        s_after records: a sweep proposes each spin once, so spin path[j]
        differs between s_before and s_after iff proposal j was accepted.
        Per proposal, at the state the recorded decisions lead to: r2 =
        (psi(s')/psi(s))^2 in FP64, the uniform u, the recorded decision and
        the rule's (u < r2).  Returns (r2, u, taken, rule, states) with arrays
        [B][N] (proposal order) and states[B][N][N] the configuration each
        proposal starts from."""
        s0 = np.ascontiguousarray(s_before, dtype=np.uint8)
        s1 = np.ascontiguousarray(s_after, dtype=np.uint8)
        B, N = s0.shape
        r2 = np.empty((B, N))
        u = np.empty((B, N))
        taken = np.zeros((B, N), dtype=bool)
        states = np.empty((B, N, N), dtype=np.uint8)

        def run(c):
            s = s0[c].copy()
            m, e = self.amplitude(s)
            for j in range(N):
                i = int(self.path[j])
                states[c, j] = s
                mf, ef = self.flip_amplitude(s, i)
                d = ef - e
                r = math.ldexp(mf / m, d) if (m != 0.0 and d < 1000) else math.inf
                r2[c, j] = r * r
                u[c, j] = mcmc_uniform(seed, chain0 + c, sweep, j)
                taken[c, j] = s1[c, i] != s0[c, i]
                if taken[c, j]:
                    s[i] ^= 1
                    m, e = mf, ef
        if threads <= 1 or B < 2:
            for c in range(B):
                run(c)
        else:
            with ThreadPoolExecutor(min(threads, B)) as ex:
                list(ex.map(run, range(B)))
        return r2, u, taken, u < r2, states


def mps_energy(inst) -> float:
    """<psi|H|psi> / <psi|psi> of an R = 1 RTT -- a matrix product state in the
    order of its path (Sec. 2.1, MPS = TT with Omega = N) -- by double-layer
    transfer matrices, polynomial in N and chi: E <- sum_{s,t} O(s,t)
    A_k[s]^T E A_k[t] site by site from b_L b_L^T, closed with b_R, each
    contraction rescaled by its largest entry (the scales summed as logs); one
    pass per Hamiltonian term, divided by the pass without operators."""
    n, path, A = inst.n_spins, np.asarray(inst.path), np.asarray(inst.tensors)
    if path.shape[0] != n:
        raise ValueError("mps_energy needs R = 1 (each spin on one site)")
    pos = {int(path[k]): k for k in range(path.shape[0])}
    Zd = np.array([[1.0, 0.0], [0.0, -1.0]])
    Xo = np.array([[0.0, 1.0], [1.0, 0.0]])

    def expval(ops_at_sites):
        E = np.outer(inst.b_left, inst.b_left)
        logs = 0.0
        for k in range(path.shape[0]):
            O = ops_at_sites.get(k)
            En = np.zeros_like(E)
            for s in (0, 1):
                for t in (0, 1):
                    w = (1.0 if s == t else 0.0) if O is None else O[s, t]
                    if w != 0.0:
                        En += w * (A[k, s].T @ E @ A[k, t])
            mx = np.abs(En).max()
            E = En / mx
            logs += math.log(mx)
        return float(inst.b_right @ E @ inst.b_right), logs

    den, ld = expval({})
    e = 0.0
    for i, j in np.asarray(inst.bonds).reshape(-1, 2):
        num, ln = expval({pos[int(i)]: Zd, pos[int(j)]: Zd})
        e += inst.J * num / den * math.exp(ln - ld)
    for i in range(n):
        num, ln = expval({pos[i]: Xo})
        e -= inst.h * num / den * math.exp(ln - ld)
    return e


def philox4x64(counter, key):
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    lib.orc_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform_keyed(seed, stream, c0, c1, c2):
    return _load().orc_uniform_keyed(int(seed), int(stream), int(c0), int(c1), int(c2))


def mcmc_uniform(seed, chain, sweep, proposal):
    return _load().orc_mcmc_uniform(int(seed), int(chain), int(sweep), int(proposal))


# ---------------------------------------------------------------------------
# Statistics of a local-energy trace x[T][B] (plain numpy, FP64)
# ---------------------------------------------------------------------------

def autocorrelation(x: np.ndarray, max_lag: int) -> np.ndarray:
    """Chain-averaged normalised autocorrelation rho(t), t = 0..max_lag.

    C(t) = mean over chains c of (1/(T-t)) sum_s (x_{s,c}-m_c)(x_{s+t,c}-m_c),
    m_c the chain mean; rho(t) = C(t)/C(0)."""
    T, B = x.shape
    d = x - x.mean(axis=0, keepdims=True)
    c = np.empty(max_lag + 1)
    for t in range(max_lag + 1):
        c[t] = np.mean(np.sum(d[: T - t] * d[t:], axis=0) / (T - t))
    if c[0] <= 0:
        return np.zeros_like(c)
    return c / c[0]


def tau_int(x: np.ndarray, c_window: float = 5.0) -> tuple[float, int]:
    """Sokal's automatic window: tau(W) = 1/2 + sum_{t=1..W} rho(t); W* is the
    smallest W >= 1 with W >= c * tau(W).  Returns (tau(W*), W*)."""
    T, _ = x.shape
    if T < 2:
        return 0.5, 0
    rho = autocorrelation(x, T - 1)
    tau = 0.5
    for W in range(1, T):
        tau += rho[W]
        if W >= c_window * tau:
            return max(tau, 0.5), W
    return max(tau, 0.5), T - 1


def observables(trace: np.ndarray, n_spins: int, n_accept=None, n_proposals_per_chain=None,
                c_window: float = 5.0) -> dict:
    """mean, var (1/n), tau_int, ess = n/(2 tau), se = sqrt(var*2tau/n),
    se_bin (bins of length ceil(20 tau) per chain, <= T), se_chain (chain
    means), v_score = N var / mean^2, accept_rate."""
    x = np.asarray(trace, dtype=np.float64)
    T, B = x.shape
    n = T * B
    mean = float(x.mean())
    var = float(np.mean((x - mean) ** 2))
    tau, W = tau_int(x, c_window)
    ess = n / (2.0 * tau)
    se = math.sqrt(var * 2.0 * tau / n) if n > 0 else float("nan")
    lb = int(min(T, max(1, math.ceil(20.0 * tau))))
    nb = T // lb
    if nb >= 1 and nb * B >= 2:
        bm = x[: nb * lb].reshape(nb, lb, B).mean(axis=1).ravel()
        se_bin = float(np.std(bm, ddof=1) / math.sqrt(bm.size))
    else:
        se_bin = float("nan")
    cm = x.mean(axis=0)
    se_chain = float(np.std(cm, ddof=1) / math.sqrt(B)) if B >= 2 else float("nan")
    acc = float("nan")
    if n_accept is not None and n_proposals_per_chain:
        acc = float(np.sum(n_accept)) / (B * float(n_proposals_per_chain))
    return dict(mean=mean, var=var, tau_int=tau, window=W, ess=ess, se=se, se_bin=se_bin,
                se_chain=se_chain, v_score=n_spins * var / mean ** 2 if mean != 0 else float("inf"),
                accept_rate=acc, n=n)
